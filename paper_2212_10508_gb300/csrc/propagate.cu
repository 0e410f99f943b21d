// Batched propagation of parareal intervals and the parareal correction sweep.
//
//  * FINE (SNAP): one persistent cooperative kernel runs every member's sub-steps.  Members
//    are sorted by their number of steps (longest first) so that the members still active at
//    sub-step l form a prefix.  Each sub-step has two phases: (A) neighbour lists and pair
//    derivatives dE_i/dr_ik of the active atoms (FP32: batches of up to 32 atoms per CTA; FP64:
//    one warp per atom), (B) the force gather and the Langevin update.  The FP32 path runs them
//    as a dataflow schedule with per-member dependencies (fine_flow), the FP64 path with bounded
//    grid barriers between the phases (fine_loop).  Uneven interval lengths cost nothing beyond
//    the active prefix.
//  * COARSE (Finnis-Sinclair EAM, or SNAP of band limit 2J = 2 for Strategy I): one CTA per
//    member runs the whole interval in shared memory.
//  * parareal_correct: one CTA walks the window sequentially (Algorithm 2's inner loop) with
//    the same per-CTA coarse code, so C(cur_n) here equals C(prev_n) of the batched path bit
//    for bit when the states are equal.
#include <algorithm>

#include "eam_device.cuh"
#include "langevin_device.cuh"
#include "pmd_internal.h"
#include "snap_coarse.cuh"
#include "snap_kernels.cuh"

namespace pmd {

SnapView snap_view(const pmd_snap* s, const double* beta);
int snap_reserve_impl(pmd_snap* s, long na);

constexpr int COARSE_MAX_THREADS = 512;   // one CTA per SM, up to 128 registers per thread

// ---- host-side parameter packing -----------------------------------------------------------
LangevinDev make_langevin(const pmd_langevin& lp) {
    LangevinDev L{};
    const double kT_m = KB * lp.T / lp.mass * FTOA;
    const double f2a = FTOA / lp.mass;
    L.dt = lp.dt;
    L.hdt = 0.5 * lp.dt;
    L.hdf = 0.5 * lp.dt * f2a;
    L.hdg = 0.5 * lp.dt * lp.gamma;
    for (int C = 0; C < 4; ++C) L.sig[C] = 0.5 * std::sqrt(2.0 * lp.gamma * kT_m * (double)C * lp.dt);
    L.c1 = std::exp(-lp.gamma * lp.dt);
    L.c2 = std::sqrt(kT_m * (1.0 - L.c1 * L.c1));
    L.scheme = lp.scheme;
    L.schedule = lp.schedule;
    L.seed = lp.seed;
    return L;
}

FSDev make_fs(const pmd_fs_params& p) {
    FSDev f{p.d, p.A, p.c, p.c0, p.c1, p.c2, 0.f};
    const double rm = std::max(p.d, p.c) + 1e-3;
    f.screen2 = (float)(rm * rm);
    return f;
}

// ---- FINE: persistent cooperative kernel ---------------------------------------------------
struct FineArgs {
    SnapView v;
    int nbatch, n;
    double box0, box1, box2;
    double* q;
    double* vel;
    long stride;
    const int32_t* nsteps;
    const int64_t* ids;
    LangevinDev L;
    // scratch
    int* nbr;
    int* nnb;
    void* dedr;
    float4* qf;
    double* vh;
    const int* order;     // members sorted by nsteps, longest first
    const int* Ls;        // nsteps in that order
    const int* Lmax;
    unsigned int* bar;
    int* status;
    double* gstep;          // FP32 path: G_{ell} of the sub-step's items [item][3], drawn in phase A
    unsigned char* pos;     // reverse-slot tables [member][n][n], or nullptr (binary search)
    SBShape shape;          // FP32 path: run-time shape of the batched pass
    int b_group;            // atoms per warp in phase B (1..SB_B_GROUP_MAX)
    int merge_b;            // FP32 path: large sub-steps run phase B on the CTA completing a member
    unsigned long long* flow;   // FP32 path (64-bit words, no wrap for any launch): [0] next item, [1] abort,
                                //   [2, 2 + nbatch) atoms done in phase A
                            // per member (order position), [2 + nbatch, 2 + 2 nbatch) in phase B
};

__global__ void k_fine_prologue(const int32_t* __restrict__ nsteps, int nbatch, int schedule, int* __restrict__ order,
                                int* __restrict__ Ls, int* __restrict__ Lmax, int* status) {
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nbatch; b += blockDim.x) {
        int Lb = nsteps[b];
        if (Lb < 0 || (schedule == PMD_SCHED_L1_SYM && Lb > 1)) {
            flag(status, ST_BADARG);
            Lb = 0;
        }
        int rank = 0;
        for (int c = 0; c < nbatch; ++c) {
            int Lc = nsteps[c];
            if (Lc < 0 || (schedule == PMD_SCHED_L1_SYM && Lc > 1)) Lc = 0;
            rank += (Lc > Lb) || (Lc == Lb && c < b);
        }
        order[rank] = b;
        Ls[rank] = Lb;
        atomicMax(&s_max, Lb);
    }
    __syncthreads();
    if (threadIdx.x == 0) *Lmax = s_max;
}

__global__ void k_wrap_members(const double* __restrict__ q, long stride, int nbatch, int n, double b0, double b1,
                               double b2, float4* __restrict__ qf) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nbatch * n) return;
    const long m = idx / n;
    const int i = (int)(idx % n);
    const double* Q = q + m * stride;
    const double box[3] = {b0, b1, b2};
    qf[idx] = wrap_f32(Q[i], Q[n + i], Q[2 * n + i], box);
}

// number of members with at least max(ell, 1) steps (Ls sorted descending)
__device__ __forceinline__ int active_members(const int* Ls, int nbatch, int ell) {
    const int need = ell < 1 ? 1 : ell;
    int lo = 0, hi = nbatch;   // first index with Ls < need
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (Ls[mid] >= need) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Phase B of sub-step ell for the items it = first + r * stride, r < group, it < items, one
// warp: the noise G_{ell,n} of all the group's atoms (FP32 path: drawn during phase A and read
// from gstep; FP64 path: lanes 2r and 2r+1 draw Philox blocks 0 and 1 of atom r: G_x, G_y and
// G_z), the force gather of each atom (whole warp, lanes = neighbour slots), and the Langevin
// update of all atoms at once (lane 3r + al advances component al of atom r).  Positions and
// velocities are loaded before the gathers.
constexpr int SB_B_GROUP_MAX = 10;   // 3 lanes per atom for the update

template <typename real>
__device__ __noinline__ void fine_phase_b(const FineArgs& a, long first, long stride, long items, int ell, int lane) {
    const int SB_B_GROUP = a.b_group;
    const int n = a.n;
    const LangevinDev& Lp = a.L;
    const double box[3] = {a.box0, a.box1, a.box2};
    // this lane's roles: noise for atom rn = lane >> 1 (block lane & 1), update of atom ru = lane / 3
    const int rn = lane >> 1, ru = lane / 3, al = lane - 3 * ru;
    const long itn = first + (long)rn * stride, itu = first + (long)ru * stride;
    double g0 = 0.0, g1 = 0.0;
    if (sizeof(real) == 8 && rn < SB_B_GROUP && itn < items) {   // FP32 path: drawn in phase A
        const int m = a.order[itn / n], k = (int)(itn % n);
        const int L = a.nsteps[m] < 0 ? 0 : a.nsteps[m];
        if (Lp.scheme == PMD_SCHEME_PAPER || ell < L) {
            const uint64_t un = (uint64_t)a.ids[m];
            uint32_t c[4] = {2u * (uint32_t)k + (uint32_t)(lane & 1), (uint32_t)ell, (uint32_t)un, (uint32_t)(un >> 32)};
            philox4x32_10(c, (uint32_t)Lp.seed, (uint32_t)(Lp.seed >> 32));
            box_muller(c, g0, g1);
        }
    }
    // update lanes: state of component al of atom ru
    const bool upd = ru < SB_B_GROUP && itu < items;
    int mu = 0, ku = 0, Lu = 0;
    double qv = 0.0, vv = 0.0, vhv = 0.0;
    long e = 0;
    if (upd) {
        mu = a.order[itu / n];
        ku = (int)(itu % n);
        Lu = a.nsteps[mu] < 0 ? 0 : a.nsteps[mu];
        e = (long)al * n + ku;
        qv = a.q[mu * a.stride + e];
        vv = a.vel[mu * a.stride + e];
        vhv = a.vh[(long)mu * 3 * n + e];
    }
    // gathers, one atom at a time; lane 3r + al keeps component al of atom r
    double Fa = 0.0;
    FF Ff{0.f, 0.f};
    for (int r = 0; r < SB_B_GROUP; ++r) {
        const long it = first + (long)r * stride;
        if (it >= items) break;
        const int m = a.order[it / n], k = (int)(it % n);
        const unsigned char* pos = a.pos ? a.pos + (size_t)m * n * n : nullptr;
        if constexpr (sizeof(real) == 4) {   // double-float sums; hi + lo evaluated by the update lane
            FF F[3];
            warp_gather_force_ff(a.nbr + (long)m * n * NMAX, a.nnb + (long)m * n,
                                 (const float*)a.dedr + (long)m * n * NMAX * 3, k, lane, F, a.status, pos, n);
            if (ru == r) Ff = al == 0 ? F[0] : (al == 1 ? F[1] : F[2]);
        } else {
            double F[3];
            warp_gather_force<real>(a.nbr + (long)m * n * NMAX, a.nnb + (long)m * n,
                                    (const real*)a.dedr + (long)m * n * NMAX * 3, k, lane, F, a.status, pos, n);
            if (ru == r) Fa = al == 0 ? F[0] : (al == 1 ? F[1] : F[2]);
        }
    }
    if (sizeof(real) == 4) Fa = (double)Ff.hi + (double)Ff.lo;
    // G of (ru, al): G_x, G_y from lane 2 ru, G_z from lane 2 ru + 1
    const int src = 2 * (ru < SB_B_GROUP ? ru : 0) + (al == 2 ? 1 : 0);
    const double s0 = __shfl_sync(0xffffffffu, g0, src), s1 = __shfl_sync(0xffffffffu, g1, src);
    double G = al == 1 ? s1 : s0;
    if (sizeof(real) == 4 && upd) G = a.gstep[itu * 3 + al];
    double qn = qv;
    if (upd) {
        bool bad = false;
        double* Q = a.q + mu * a.stride;
        double* V = a.vel + mu * a.stride;
        double* VH = a.vh + (long)mu * 3 * n;
        if (Lp.scheme == PMD_SCHEME_PAPER) {
            const double s = sched_sigma(Lp, ell);
            double v = vv;
            const double vh = ell == 0 ? v : vhv;
            if (ell > 0) v = half_kick(Lp, vh, Fa, vh, s, G);           // finish step ell-1
            if (ell < Lu) {
                const double vhn = half_kick(Lp, v, Fa, vh, s, G);      // first half of step ell
                qn = drift(qv, Lp.dt, vhn);
                if (!isfinite(qn)) bad = true;
                if (fabs(qn - qv) > 0.5 * box[al]) flag(a.status, ST_LOSTATOM);
                Q[e] = qn;
                VH[e] = vhn;
            }
            V[e] = v;
        } else {
            double v = vv;
            if (ell > 0) v = kick_b(Lp, v, Fa);
            if (ell < Lu) {
                double q = qv;
                v = kick_b(Lp, v, Fa);
                q = __dadd_rn(q, __dmul_rn(Lp.hdt, v));
                v = ou_o(Lp, v, G);
                q = __dadd_rn(q, __dmul_rn(Lp.hdt, v));
                if (!isfinite(q)) bad = true;
                if (fabs(q - qv) > 0.5 * box[al]) flag(a.status, ST_LOSTATOM);
                Q[e] = q;
                qn = q;
            }
            V[e] = v;
        }
        if (bad) flag(a.status, ST_NONFINITE);
    }
    // wrapped FP32 copy of the new position (lane 3r assembles the three components)
    const double qy = __shfl_down_sync(0xffffffffu, qn, 1), qz = __shfl_down_sync(0xffffffffu, qn, 2);
    if (sizeof(real) == 4 && upd && al == 0 && ell < Lu) a.qf[(long)mu * n + ku] = wrap_f32(qn, qy, qz, box);
}

// Phase A of sub-step ell over the items (active member, atom) = [0, A n).
// Draws G_{ell,n} of the batch's items [bs, bs + na) into gstep: task t = 32 w + lane of the first
// warps, atom slot t / 2, Philox block t % 2 (block 0 gives G_x, G_y, block 1 G_z).
struct FineNoiseSide {
    const FineArgs* a;
    long bs;
    int na, ell;
    __device__ void operator()(int warp, int lane) const {
        const int t = warp * 32 + lane;
        if (warp * 32 >= 2 * na || t >= 2 * na) return;
        const int n = a->n;
        const long it = bs + (t >> 1);
        const int m = a->order[it / n], k = (int)(it % n), blk = t & 1;
        const uint64_t un = (uint64_t)a->ids[m];
        uint32_t c[4] = {2u * (uint32_t)k + (uint32_t)blk, (uint32_t)ell, (uint32_t)un, (uint32_t)(un >> 32)};
        philox4x32_10(c, (uint32_t)a->L.seed, (uint32_t)(a->L.seed >> 32));
        double g0, g1;
        box_muller(c, g0, g1);
        if (blk == 0) {
            a->gstep[it * 3 + 0] = g0;
            a->gstep[it * 3 + 1] = g1;
        } else {
            a->gstep[it * 3 + 2] = g0;
        }
    }
};

// FP64 path: warp per atom over the grid, grid barriers between the phases
template <typename real, int TJ, class SH>
__device__ __forceinline__ void fine_phase_a(const FineArgs& a, const SH& sh, long items, const double box[3], int ell) {
    const int n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long gwarp = (long)blockIdx.x * wpb + warp, nwarps = (long)gridDim.x * wpb;
    for (long it = gwarp; it < items; it += nwarps) {
        const int m = a.order[it / n];
        const int i = (int)(it % n);
        real* dd = (real*)a.dedr + ((long)m * n + i) * NMAX * 3;
        snap_atom_warp2<real, TJ>(sh.ws[warp], sh.tab, a.v.yt, sh.cg, sh.beff, a.v.sp, lane, n, i, a.q + m * a.stride,
                                  a.qf + (long)m * n, box, a.nbr + ((long)m * n + i) * NMAX, a.nnb + (long)m * n + i,
                                  dd, nullptr, a.status);
    }
}

template <typename real, int TJ, class SH>
__device__ __forceinline__ void fine_loop(const FineArgs& a, const SH& sh) {
    const int lane = threadIdx.x & 31;
    const long gwarp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const int n = a.n;
    const double box[3] = {a.box0, a.box1, a.box2};
    const GridBarrier gb{a.bar, gridDim.x};
    const int Lmax = *a.Lmax;
    for (int ell = 0; ell <= Lmax; ++ell) {
        const int A = active_members(a.Ls, a.nbatch, ell);
        if (A == 0) break;
        const long items = (long)A * n;
        fine_phase_a<real, TJ>(a, sh, items, box, ell);
        if (!grid_sync(gb, a.status, ST_TIMEOUT)) return;
        for (long first = gwarp; first < items; first += (long)a.b_group * nwarps)
            fine_phase_b<real>(a, first, nwarps, items, ell, lane);
        if (!grid_sync(gb, a.status, ST_TIMEOUT)) return;
    }
}

// ---- FP32 path: dataflow schedule of the sub-steps ------------------------------------------
// The work of a launch is a fixed sequence of items: for each sub-step ell, the phase-A batches
// (bA consecutive items of the sub-step's active sequence, the last one partial) and then the
// phase-B groups (bB consecutive items).  bA = min(SB_ATOMS, ceil(items / CTAs)) and bB =
// min(16 b_group, ceil(items / CTAs)): a small sub-step is spread over all CTAs (short items on
// the critical path of one system), a large one is cut into full batches.  CTAs take items from a global counter, in
// that order, and an item waits only for the members it touches: phase A of ell > 0 for all
// phase-B work of its members at ell - 1 (their positions are then final, and so is every read of
// the per-step arrays it overwrites), phase B of ell for all phase-A work of its members at ell
// (pair derivatives, neighbour lists and Gaussian increments).  Members are independent systems,
// so a CTA that finishes early goes on with other members' work instead of idling at a grid
// barrier.  Every wait is for items earlier in the sequence and all CTAs are resident (cooperative
// launch): the earliest unfinished item never waits, so the schedule cannot deadlock.  No atom's
// arithmetic depends on the batch it lands in, so the results are those of any other schedule.
struct FlowCursor {
    int ell = 0, A = 0;    // sub-step of the window and its active members
    long base = 0;         // first item of the sub-step
    long nA = 0, nB = 0;   // its phase-A and phase-B items
    long bA = 1, bB = 1;   // and their sizes in atoms
    int merged = 0;        // phase B run by the CTA that completes a member's phase A (no B items)
};

// A sub-step with at least one full wave of full batches runs each member's phase B on the CTA
// whose batch completes the member's phase A (no phase-B items: no CTA takes a B item and waits
// for a batch still running elsewhere); smaller sub-steps keep B items spread over the CTAs, which
// keeps the chain A -> B -> A of few members short.
__device__ __forceinline__ void flow_set(const FineArgs& a, FlowCursor& c, int bmax) {
    c.A = c.ell <= *a.Lmax ? active_members(a.Ls, a.nbatch, c.ell) : 0;
    const long items = (long)c.A * a.n;
    const long per = (items + gridDim.x - 1) / gridDim.x;
    c.bA = per < SB_ATOMS ? (per > 0 ? per : 1) : SB_ATOMS;
    c.bB = per < bmax ? (per > 0 ? per : 1) : bmax;
    c.merged = a.merge_b && items >= (long)gridDim.x * SB_ATOMS;
    c.nA = (items + c.bA - 1) / c.bA;
    c.nB = c.merged ? 0 : (items + c.bB - 1) / c.bB;
}

// Thread 0: wait until *ctr >= target (bounded; one item takes < 1 ms, the limit ~4 s; the abort
// word ends every wait of the launch).
__device__ __forceinline__ bool flow_wait(const FineArgs& a, unsigned long long* ctr, unsigned long long target) {
    return bounded_wait_geq(ctr, target, a.flow + 1, a.status, ST_TIMEOUT);
}

// Self-test of the bounded waits: one CTA waits on a 64-bit counter that nothing increments (the
// dataflow schedule's wait), then on a 32-bit one, then on a grid barrier of two CTAs with only
// itself launched (the FP64 path's barrier); each must give up after `polls` polls with
// ST_TIMEOUT.  w64: [0] counter, [1] abort word; w32: [0] counter, [1] abort word, [2..5]
// barrier words.
__global__ void k_selftest_waits(unsigned long long* w64, unsigned int* w32, int* status, long long polls) {
    if (threadIdx.x == 0) {
        bounded_wait_geq<unsigned long long>(w64, 1ull, w64 + 1, status, ST_TIMEOUT, polls);
        bounded_wait_geq<unsigned int>(w32, 1u, w32 + 1, status, ST_TIMEOUT, polls);
    }
    __syncthreads();
    const GridBarrier gb{w32 + 2, 2u};
    grid_sync(gb, status, ST_TIMEOUT, polls);
}

int selftest_waits(pmd_engine* e, long long polls, cudaStream_t st) {
    int rc;
    if ((rc = e->s_selftest.ensure(8 * sizeof(unsigned long long)))) return rc;
    unsigned long long* w64 = e->s_selftest.as<unsigned long long>();   // [0, 2): 64-bit words
    unsigned int* w32 = reinterpret_cast<unsigned int*>(w64 + 2);        // [2, 8): 32-bit words
    PMD_CUDA_TRY(cudaMemsetAsync(w64, 0, 8 * sizeof(unsigned long long), st));
    k_selftest_waits<<<1, 32, 0, st>>>(w64, w32, e->status.as<int>(), polls);
    PMD_CUDA_TRY(cudaGetLastError());
    return PMD_OK;
}

template <int TJ>
__device__ void fine_flow(const FineArgs& a, const SBShared<TJ>& sh) {
    __shared__ long s_item[5];   // sub-step, phase (0 A, 1 B, -1 done), items [first, end), merged B
    __shared__ int s_comp[SB_ATOMS + 2];   // merged mode: members whose phase A this item completed
    const int n = a.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int bmax = nw * a.b_group;   // phase-B item: at most b_group atoms per warp
    const double box[3] = {a.box0, a.box1, a.box2};
    unsigned long long* doneA = a.flow + 2;
    unsigned long long* doneB = a.flow + 2 + a.nbatch;
    FlowCursor c;   // thread 0's view of the sequence (items are taken in increasing order)
    if (threadIdx.x == 0) flow_set(a, c, bmax);
    for (;;) {
        if (threadIdx.x == 0) {
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> head(a.flow[0]), ab(a.flow[1]);
            const long t = ab.load(cuda::memory_order_relaxed) != 0 ? -1 : (long)head.fetch_add(1ull, cuda::memory_order_relaxed);
            while (t >= 0 && c.A > 0 && t >= c.base + c.nA + c.nB) {
                c.base += c.nA + c.nB;
                ++c.ell;
                flow_set(a, c, bmax);
            }
            const long items = (long)c.A * n;
            int ph = -1;
            long s = 0, e = 0;
            if (t >= 0 && c.A > 0) {
                const long r = t - c.base;
                ph = r < c.nA ? 0 : 1;
                s = ph == 0 ? r * c.bA : (r - c.nA) * c.bB;
                e = s + (ph == 0 ? c.bA : c.bB);
                if (e > items) e = items;
            }
            // wait for the members of [s, e): A of ell > 0 on their phase B of ell - 1, B on their phase A
            bool ok = true;
            if (ph >= 0 && !(ph == 0 && c.ell == 0)) {
                for (long p = s / n; p <= (e - 1) / n && ok; ++p)
                    ok = ph == 0 ? flow_wait(a, doneB + p, (unsigned long long)c.ell * n)
                                 : flow_wait(a, doneA + p, (unsigned long long)(c.ell + 1) * n);
            }
            s_item[0] = c.ell;
            s_item[1] = ok ? ph : -1;
            s_item[2] = s;
            s_item[3] = e;
            s_item[4] = c.merged;
        }
        __syncthreads();
        const int ell = (int)s_item[0];
        const int ph = (int)s_item[1];
        const long s = s_item[2], e = s_item[3];
        const bool merged = s_item[4] != 0;
        if (ph < 0) return;
        // both branches end with a CTA barrier, after which thread 0 may rewrite s_item
        if (ph == 0) {
            const int na = (int)(e - s);
            auto at = [&](int slot) {
                const long it = s + slot;
                const long m = a.order[it / n];
                const int i = (int)(it % n);
                const long ai = m * n + i;
                return SBAtom{a.q + m * a.stride, a.qf + m * n, i, a.nbr + ai * NMAX, a.nnb + ai,
                              (float*)a.dedr + ai * NMAX * 3, nullptr,
                              a.pos ? a.pos + ((size_t)m * n + i) * n : nullptr};
            };
            const FineNoiseSide side{&a, s, na, ell};
            sb_batch<TJ>(sh, sb_tables(a.v), a.v.sp, na, at, n, box, a.status, true, side, a.shape);   // ends with a barrier
        } else {
            if (s + warp < e) fine_phase_b<float>(a, s + warp, nw, e, ell, lane);
            __syncthreads();
        }
        if (!merged) {
            if (threadIdx.x == 0) {   // publish: the item's atoms per member
                unsigned long long* done = ph == 0 ? doneA : doneB;
                for (long p = s / n; p <= (e - 1) / n; ++p) {
                    const long lo = p * n > s ? p * n : s, hi = (p + 1) * n < e ? (p + 1) * n : e;
                    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> x(done[p]);
                    x.fetch_add((unsigned long long)(hi - lo), cuda::memory_order_release);
                }
            }
            continue;
        }
        // merged sub-step: publish the phase-A atoms; the CTA that completes a member (its count
        // reaches (ell + 1) n, acquire: every batch of the member is visible) runs the member's
        // phase B at once and publishes it
        if (threadIdx.x == 0) {
            int k = 0;
            for (long p = s / n; p <= (e - 1) / n; ++p) {
                const long lo = p * n > s ? p * n : s, hi = (p + 1) * n < e ? (p + 1) * n : e;
                cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> x(doneA[p]);
                const unsigned long long old = x.fetch_add((unsigned long long)(hi - lo), cuda::memory_order_acq_rel);
                if (old + (unsigned long long)(hi - lo) == (unsigned long long)(ell + 1) * n) s_comp[1 + k++] = (int)p;
            }
            s_comp[0] = k;
        }
        __syncthreads();
        const int ncomp = s_comp[0];
        for (int c2 = 0; c2 < ncomp; ++c2) {
            const long p = s_comp[1 + c2];
            const long b0 = p * n, b1 = b0 + n;
            for (long base = b0; base < b1; base += (long)nw * a.b_group)
                if (base + warp < b1) fine_phase_b<float>(a, base + warp, nw, b1, ell, lane);
            __syncthreads();
            if (threadIdx.x == 0) {
                cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> x(doneB[p]);
                x.fetch_add((unsigned long long)n, cuda::memory_order_release);
            }
        }
    }
}

template <typename real, int TJ, int NTH = snap_cta_threads<real, TJ>()>
__global__ void __launch_bounds__(NTH, 1) k_fine_persistent(FineArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (sizeof(real) == 4) {
        SBShared<TJ> sh = sb_shared_carve<TJ>(smem, a.v);
        sb_shared_load<TJ>(sh, a.v);
        __syncthreads();
        fine_flow<TJ>(a, sh);
    } else {
        SnapShared<real, TJ> sh = snap_shared_carve<real, TJ>(smem, a.v);
        snap_shared_load<real, TJ>(sh, a.v);
        __syncthreads();
        fine_loop<real, TJ>(a, sh);
    }
}

template <typename real, int TJ>
static int launch_fine(pmd_engine* e, int nbatch, int n, double* q, double* v, long stride, const int32_t* nsteps,
                       const int64_t* ids, const pmd_langevin& lp, cudaStream_t st) {
    pmd_snap* s = e->snap;
    FineArgs a{};
    a.v = snap_view(s, e->beta.as<double>());
    a.nbatch = nbatch;
    a.n = n;
    a.box0 = e->p.box[0];
    a.box1 = e->p.box[1];
    a.box2 = e->p.box[2];
    a.q = q;
    a.vel = v;
    a.stride = stride;
    a.nsteps = nsteps;
    a.ids = ids;
    a.L = make_langevin(lp);
    a.nbr = e->s_nbr.as<int>();
    a.nnb = e->s_nnb.as<int>();
    a.dedr = e->s_dedr.p;
    a.qf = e->s_qf.as<float4>();
    a.vh = e->s_vh.as<double>();
    a.gstep = e->s_gstep.as<double>();
    a.shape.rows2_atoms = e->tune.rows2_atoms;
    a.shape.rows4_atoms = e->tune.rows4_atoms;
    a.shape.noise_stage = e->tune.noise_stage;
    a.b_group = e->tune.b_group < 1 ? 1 : (e->tune.b_group > SB_B_GROUP_MAX ? SB_B_GROUP_MAX : e->tune.b_group);
    a.merge_b = 1;
    a.pos = n <= PMD_POS_TABLE_MAX_ATOMS && sizeof(real) == 4 ? e->s_pos.as<unsigned char>() : nullptr;
    a.order = e->s_order.as<int>();
    a.Ls = e->s_order.as<int>() + e->cap_batch;
    a.Lmax = e->s_order.as<int>() + 2 * e->cap_batch;
    unsigned int* words = reinterpret_cast<unsigned int*>(e->status.as<int>() + 1);
    a.bar = words;
    a.status = e->status.as<int>();
    a.flow = e->s_flow.as<unsigned long long>();
    PMD_CUDA_TRY(cudaMemsetAsync(words, 0, 4 * sizeof(unsigned int), st));
    if (sizeof(real) == 4)
        PMD_CUDA_TRY(cudaMemsetAsync(a.flow, 0, (2 * (size_t)nbatch + 2) * sizeof(unsigned long long), st));
    k_fine_prologue<<<1, 1024, 0, st>>>(nsteps, nbatch, lp.schedule, e->s_order.as<int>(), (int*)a.Ls, (int*)a.Lmax,
                                        a.status);
    PMD_CUDA_TRY(cudaGetLastError());
    if (sizeof(real) == 4) {
        const long na = (long)nbatch * n;
        k_wrap_members<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(q, stride, nbatch, n, a.box0, a.box1, a.box2,
                                                                     a.qf);
        PMD_CUDA_TRY(cudaGetLastError());
    }
    // FP32, 2J = 8: the CTA size is a tuning knob (16 warps, or 8 with twice the registers)
    const bool half = sizeof(real) == 4 && TJ == 8 && e->tune.warps == 8;
    const int threads = half ? SB_THREADS / 2 : snap_cta_threads<real, TJ>();
    const size_t sm = sizeof(real) == 4 ? sb_shared_bytes<TJ>(a.v) : snap_shared_bytes<real, TJ>(a.v, threads / 32);
    void (*kern)(FineArgs) = k_fine_persistent<real, TJ>;
    if constexpr (sizeof(real) == 4 && TJ == 8)
        if (half) kern = k_fine_persistent<real, TJ, SB_THREADS / 2>;
    PMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    PMD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm));
    if (per_sm < 1) return fail(PMD_EUNSUPPORTED, "persistent SNAP kernel does not fit on an SM");
    const int grid = per_sm * e->num_sms;
    void* args[] = {&a};
    // inside a stream capture the timing events must become event nodes of the graph
    unsigned int ev_flags = cudaEventRecordDefault;
    if (e->profile) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PMD_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusActive) ev_flags = cudaEventRecordExternal;
        PMD_CUDA_TRY(cudaEventRecordWithFlags(e->ev0, st, ev_flags));
    }
    PMD_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(threads), args, sm, st));
    if (e->profile) {
        PMD_CUDA_TRY(cudaEventRecordWithFlags(e->ev1, st, ev_flags));
        e->prof_recorded = 1;
    }
    return PMD_OK;
}

int fine_propagate(pmd_engine* e, int nbatch, int n, double* q, double* v, long stride, const int32_t* nsteps,
                   const int64_t* ids, const pmd_langevin& lp, cudaStream_t st) {
    const bool f64 = e->p.fine.precision == PMD_FP64;
    switch (e->p.fine.twojmax) {
#define PMD_FINE_CASE(TJV)                                                                         \
    case TJV:                                                                                      \
        return f64 ? launch_fine<double, TJV>(e, nbatch, n, q, v, stride, nsteps, ids, lp, st)     \
                   : launch_fine<float, TJV>(e, nbatch, n, q, v, stride, nsteps, ids, lp, st);
        PMD_FINE_CASE(2)
        PMD_FINE_CASE(4)
        PMD_FINE_CASE(6)
        PMD_FINE_CASE(8)
#undef PMD_FINE_CASE
    }
    return fail(PMD_EUNSUPPORTED, "twojmax must be 2, 4, 6 or 8");
}

// ---- COARSE: one CTA per interval ----------------------------------------------------------
// Shared memory: q [3][n] FP64, qf [n], F [3][n], dF [n].  Velocities v and v_{l-1/2} of the
// thread's own atoms (i = tid + k*blockDim) stay in registers.
template <int KMAX>
struct OwnState {
    double v[KMAX][3];
    double vh[KMAX][3];
};

constexpr int EAM_LIST_MAX_ATOMS = 512;   // systems up to this size keep a Verlet list in shared memory
constexpr int EAM_PG_MAX_ATOMS = 256;     // ... and up to this size the FP32 pair-geometry cache

__host__ __device__ inline size_t coarse_smem_bytes(int n, bool pg = true) {
    size_t b = (size_t)n * (3 * 8 + 16 + 3 * 8 + 8) + 64;
    if (n <= EAM_LIST_MAX_ATOMS) b += (size_t)n * (EAM_LIST_CAP * 2 + 2 + 16) + 64;
    if (pg && n <= EAM_PG_MAX_ATOMS) b += (size_t)n * (EAM_PG_CAP * (16 + 2) + 2) + 64;
    return (b + 15) / 16 * 16;
}

__device__ inline EamShared coarse_carve(unsigned char* smem, int n, bool pg = true) {
    EamShared s;
    s.q = reinterpret_cast<double*>(smem);
    s.F = s.q + 3 * n;
    s.dF = s.F + 3 * n;
    s.qf = reinterpret_cast<float4*>(align_up(reinterpret_cast<size_t>(s.dF + n), 16));
    if (n <= EAM_LIST_MAX_ATOMS) {
        s.qref = s.qf + n;
        s.nbl = reinterpret_cast<unsigned short*>(s.qref + n);
        s.nbc = reinterpret_cast<unsigned char*>(s.nbl + (size_t)n * EAM_LIST_CAP);
    } else {
        s.qref = nullptr;
        s.nbl = nullptr;
        s.nbc = nullptr;
    }
    s.pg = nullptr;
    s.pj = nullptr;
    s.pgc = nullptr;
    if (pg && n <= EAM_PG_MAX_ATOMS) {
        s.pg = reinterpret_cast<float4*>(align_up(reinterpret_cast<size_t>(s.nbc + 2 * n), 16));
        s.pj = reinterpret_cast<unsigned short*>(s.pg + (size_t)n * EAM_PG_CAP);
        s.pgc = reinterpret_cast<unsigned char*>(s.pj + (size_t)n * EAM_PG_CAP);
    }
    return s;
}

// The coarse potential of the one-CTA kernels, passed by value to them: Finnis-Sinclair EAM, or
// SNAP of a small band limit (Strategy I).  setup() runs once per launch with every thread
// (tail: shared memory after the coarse state); refresh() keeps the Verlet list valid; forces()
// fills s.F.  Both end with a CTA barrier.
struct CoarseFS {
    static constexpr bool PG = true;   // uses the FP32 pair-geometry cache of the EAM passes
    FSDev fs;
    __device__ __forceinline__ void setup(unsigned char*, int) {}
    __device__ __forceinline__ void refresh(const EamShared& s, int n, const double box[3], bool force,
                                            int* status) const {
        eam_refresh_list(s, n, box, fs, force, status);
    }
    template <typename real, bool ONE>
    __device__ __forceinline__ void forces(const EamShared& s, int n, const double box[3]) const {
        eam_forces_cta<real, ONE>(s, n, box, fs, nullptr);
    }
};

template <typename R, int TJ>
struct CoarseSnap {
    static constexpr bool PG = false;
    SnapCoarseDev d;
    SnapCoarseShared<R, TJ> t;
    __device__ __forceinline__ void setup(unsigned char* tail, int n) {
        t = snap_coarse_carve<R, TJ>(tail, n, d.nblk);
        snap_coarse_load<R, TJ>(t, d);
    }
    __device__ __forceinline__ void refresh(const EamShared& s, int n, const double box[3], bool force,
                                            int* status) const {
        snap_coarse_refresh_list(s, n, box, d, force, status);
    }
    template <typename real, bool ONE>
    __device__ __forceinline__ void forces(const EamShared& s, int n, const double box[3]) const {
        snap_coarse_forces_cta<R, TJ>(s, t, n, box, d);
    }
};

// G_{l,n} of atom i: from the precomputed window buffer [L+1][3][n] of this interval, or drawn
template <int KMAX>
__device__ __forceinline__ void coarse_noise(const LangevinDev& L, const double* Gpre, int64_t nid, int ell, int i,
                                             int n, double G[3]) {
    if (Gpre) {
#pragma unroll
        for (int al = 0; al < 3; ++al) G[al] = Gpre[((size_t)ell * 3 + al) * n + i];
    } else {
        normals3(L.seed, nid, ell, i, G);
    }
}

// Runs nsteps sub-steps of interval nid on the CTA-resident state (positions in s.q/s.qf,
// velocities in own.v).  All threads call it.  list_ok tracks whether the CTA's Verlet list has
// been built (it persists across intervals of a sweep).
template <typename real, int KMAX, class CP>
__device__ void coarse_interval_cta(const EamShared& s, OwnState<KMAX>& own, int n, const double box[3],
                                    const CP& pot, const LangevinDev& L, int nsteps, int64_t nid, const double* Gpre,
                                    bool& list_ok, int* status) {
    if (nsteps <= 0) return;
    // the Gaussian increments are loaded before the force evaluation that precedes their use
    double Gc[KMAX][3];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < n) coarse_noise<KMAX>(L, Gpre, nid, 0, i, n, Gc[k]);
    }
    pot.refresh(s, n, box, !list_ok, status);
    list_ok = true;
    pot.template forces<real, KMAX == 1>(s, n, box);
    bool bad = false;
    if (L.scheme == PMD_SCHEME_PAPER) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
            for (int al = 0; al < 3; ++al) own.vh[k][al] = own.v[k][al];
        for (int ell = 0; ell < nsteps; ++ell) {
            const double s0 = sched_sigma(L, ell), s1 = sched_sigma(L, ell + 1);
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                const int i = threadIdx.x + k * blockDim.x;
                if (i >= n) break;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const double vhn = half_kick(L, own.v[k][al], s.F[al * n + i], own.vh[k][al], s0, Gc[k][al]);
                    own.vh[k][al] = vhn;
                    const double q0 = s.q[al * n + i];
                    const double qn = drift(q0, L.dt, vhn);
                    if (!isfinite(qn)) bad = true;
                    if (fabs(qn - q0) > 0.5 * box[al]) flag(status, ST_LOSTATOM);
                    s.q[al * n + i] = qn;
                }
                s.qf[i] = wrap_f32(s.q[i], s.q[n + i], s.q[2 * n + i], box);
            }
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {   // G_{l+1}: this kick and the next step's
                const int i = threadIdx.x + k * blockDim.x;
                if (i < n) coarse_noise<KMAX>(L, Gpre, nid, ell + 1, i, n, Gc[k]);
            }
            __syncthreads();
            pot.refresh(s, n, box, false, status);
            pot.template forces<real, KMAX == 1>(s, n, box);
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                const int i = threadIdx.x + k * blockDim.x;
                if (i >= n) break;
#pragma unroll
                for (int al = 0; al < 3; ++al)
                    own.v[k][al] = half_kick(L, own.vh[k][al], s.F[al * n + i], own.vh[k][al], s1, Gc[k][al]);
            }
        }
    } else {
        for (int ell = 0; ell < nsteps; ++ell) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                const int i = threadIdx.x + k * blockDim.x;
                if (i >= n) break;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    double v = kick_b(L, own.v[k][al], s.F[al * n + i]);
                    const double q0 = s.q[al * n + i];
                    double q = __dadd_rn(q0, __dmul_rn(L.hdt, v));
                    v = ou_o(L, v, Gc[k][al]);
                    q = __dadd_rn(q, __dmul_rn(L.hdt, v));
                    if (!isfinite(q)) bad = true;
                    if (fabs(q - q0) > 0.5 * box[al]) flag(status, ST_LOSTATOM);
                    s.q[al * n + i] = q;
                    own.v[k][al] = v;
                }
                s.qf[i] = wrap_f32(s.q[i], s.q[n + i], s.q[2 * n + i], box);
            }
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {   // G_{l+1} for the next step
                const int i = threadIdx.x + k * blockDim.x;
                if (i < n && ell + 1 < nsteps) coarse_noise<KMAX>(L, Gpre, nid, ell + 1, i, n, Gc[k]);
            }
            __syncthreads();
            pot.refresh(s, n, box, false, status);
            pot.template forces<real, KMAX == 1>(s, n, box);
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                const int i = threadIdx.x + k * blockDim.x;
                if (i >= n) break;
#pragma unroll
                for (int al = 0; al < 3; ++al) own.v[k][al] = kick_b(L, own.v[k][al], s.F[al * n + i]);
            }
        }
    }
    if (bad) flag(status, ST_NONFINITE);
}

template <int KMAX>
__device__ void load_state(const EamShared& s, OwnState<KMAX>& own, int n, const double* q, const double* v,
                           const double box[3]) {
    for (int x = threadIdx.x; x < 3 * n; x += blockDim.x) s.q[x] = q[x];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
#pragma unroll
        for (int al = 0; al < 3; ++al) own.v[k][al] = i < n ? v[al * n + i] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.qf[i] = wrap_f32(s.q[i], s.q[n + i], s.q[2 * n + i], box);
    __syncthreads();
}

template <int KMAX>
__device__ void store_state(const EamShared& s, const OwnState<KMAX>& own, int n, double* q, double* v) {
    __syncthreads();
    for (int x = threadIdx.x; x < 3 * n; x += blockDim.x) q[x] = s.q[x];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < n) {
#pragma unroll
            for (int al = 0; al < 3; ++al) v[al * n + i] = own.v[k][al];
        }
    }
}

template <typename real, int KMAX, class CP>
__global__ void __launch_bounds__(COARSE_MAX_THREADS, 1) k_coarse_batch(int n, double b0, double b1, double b2, CP pot, LangevinDev L, double* q, double* v,
                               long stride, const int32_t* __restrict__ nsteps, const int64_t* __restrict__ ids,
                               int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const EamShared s = coarse_carve(smem, n, CP::PG);
    pot.setup(smem + coarse_smem_bytes(n, CP::PG), n);
    const double box[3] = {b0, b1, b2};
    const int m = blockIdx.x;
    int Lm = nsteps[m];
    if (Lm < 0 || (L.schedule == PMD_SCHED_L1_SYM && Lm > 1)) {
        if (threadIdx.x == 0) flag(status, ST_BADARG);
        return;
    }
    OwnState<KMAX> own;
    load_state<KMAX>(s, own, n, q + m * stride, v + m * stride, box);
    bool list_ok = false;
    coarse_interval_cta<real, KMAX>(s, own, n, box, pot, L, Lm, ids[m], nullptr, list_ok, status);
    store_state<KMAX>(s, own, n, q + m * stride, v + m * stride);
}

// Threads of the one-CTA coarse kernels (batch and sweep use the same shape, so their force sums
// are bit for bit the same): two threads per atom in the pair loops up to 256 atoms, one beyond.
static void coarse_shape(int n, int& threads, int& kmax) {
    threads = std::min(COARSE_MAX_THREADS, ((2 * n <= COARSE_MAX_THREADS ? 2 * n : n) + 31) / 32 * 32);
    kmax = (n + threads - 1) / threads;
}

// Device view of the engine's SNAP coarse context (Strategy I).
static SnapCoarseDev make_snap_coarse(const pmd_engine* e) {
    const pmd_snap* s = e->csnap;
    SnapCoarseDev d{};
    d.jobs = s->d_jobs.as<int4>();
    d.round_tb = s->d_roundtb.as<unsigned char>();
    d.cg = s->d_cg.p;
    d.beffptr = s->d_beffptr.as<int>();
    d.befft = s->d_befft.as<int>();
    d.beffc = s->d_beffc.as<double>();
    d.beta = e->cbeta.as<double>();
    d.nrounds = s->T.nrounds;
    d.ncg = (int)s->T.cg.size();
    d.nblk = (int)s->T.blk_ta.size();
    d.rcut = s->p.rcut;
    d.kappa = s->p.rfac0 * PI / s->p.rcut;
    d.switchflag = s->p.switchflag;
    const double rm = s->p.rcut + 1e-3;
    d.screen2 = (float)(rm * rm);
    return d;
}

// Calls go(kernel, potential, shared bytes) with the coarse kernel instantiation of the engine's
// coarse potential, precision and atoms per thread.
template <template <typename, int, class> class K, class Go>
static int coarse_dispatch(const pmd_engine* e, int n, int kmax, Go&& go) {
    if (e->p.coarse_kind == PMD_COARSE_SNAP) {
        if (kmax != 1 || n > EAM_LIST_MAX_ATOMS) return fail(PMD_EUNSUPPORTED, "the SNAP coarse potential supports at most 512 atoms");
        const SnapCoarseDev d = make_snap_coarse(e);
        if (e->p.coarse_snap.precision == PMD_FP64) {
            CoarseSnap<double, 2> cp{d, {}};
            return go(K<double, 1, CoarseSnap<double, 2>>::ptr(), cp,
                      coarse_smem_bytes(n, false) + snap_coarse_smem_bytes<double, 2>(n, d.ncg, d.nblk));
        }
        CoarseSnap<float, 2> cp{d, {}};
        return go(K<float, 1, CoarseSnap<float, 2>>::ptr(), cp,
                  coarse_smem_bytes(n, false) + snap_coarse_smem_bytes<float, 2>(n, d.ncg, d.nblk));
    }
    const CoarseFS cp{make_fs(e->p.coarse)};
    const bool f64 = e->p.coarse.precision == PMD_FP64;
    const size_t sm = coarse_smem_bytes(n);
    if (kmax == 1) return f64 ? go(K<double, 1, CoarseFS>::ptr(), cp, sm) : go(K<float, 1, CoarseFS>::ptr(), cp, sm);
    if (kmax == 2) return f64 ? go(K<double, 2, CoarseFS>::ptr(), cp, sm) : go(K<float, 2, CoarseFS>::ptr(), cp, sm);
    if (kmax <= 4) return f64 ? go(K<double, 4, CoarseFS>::ptr(), cp, sm) : go(K<float, 4, CoarseFS>::ptr(), cp, sm);
    return fail(PMD_EUNSUPPORTED, "coarse propagation supports at most 2048 atoms");
}

template <typename real, int KMAX, class CP>
struct CoarseBatchK {
    static auto ptr() { return &k_coarse_batch<real, KMAX, CP>; }
};

int coarse_propagate(pmd_engine* e, int nbatch, int n, double* q, double* v, long stride, const int32_t* nsteps,
                     const int64_t* ids, const pmd_langevin& lp, cudaStream_t st) {
    int threads, kmax;
    coarse_shape(n, threads, kmax);
    const LangevinDev L = make_langevin(lp);
    const double* B = e->p.box;
    auto go = [&](auto kern, auto cp, size_t sm) -> int {
        PMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<nbatch, threads, sm, st>>>(n, B[0], B[1], B[2], cp, L, q, v, stride, nsteps, ids, e->status.as<int>());
        PMD_CUDA_TRY(cudaGetLastError());
        return PMD_OK;
    };
    return coarse_dispatch<CoarseBatchK>(e, n, kmax, go);
}

// ---- parareal correction sweep ---------------------------------------------------------------
struct SweepResult {
    double delta;
    int n_stop;
    int pad;
};

// deterministic CTA-wide sum (fixed tree) of one double per thread
__device__ double cta_sum(double x, double* red) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}
__device__ double cta_max(double x, double* red) {
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

template <typename real, int KMAX, class CP>
__global__ void __launch_bounds__(COARSE_MAX_THREADS, 1) k_parareal_sweep(int n, double b0, double b1, double b2, CP pot, LangevinDev L, int nsteps, int n_in,
                                 int n_fin, const double* __restrict__ jumps, const double* __restrict__ prev,
                                 double* __restrict__ cur, double* __restrict__ cout, double delta_expl, int metric,
                                 const double* __restrict__ Gwin, SweepResult* res, int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const EamShared s = coarse_carve(smem, n, CP::PG);
    pot.setup(smem + coarse_smem_bytes(n, CP::PG), n);
    __shared__ double red[33];
    const double box[3] = {b0, b1, b2};
    const long S = 6L * n;
    OwnState<KMAX> own;
    load_state<KMAX>(s, own, n, cur, cur + 3 * n, box);
    // error sums start at n = n_in: |q^cur_{n_in} - q^prev_{n_in}| and |q^prev_{n_in}|
    double num = 0.0, den = 0.0;
    {
        double a = 0.0, b = 0.0, mx = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double d2 = 0.0;
            for (int al = 0; al < 3; ++al) {
                const double c = cur[al * n + i], p = prev[al * n + i];
                d2 += (c - p) * (c - p);
                b += p * p;
            }
            a += d2;
            mx = fmax(mx, d2);
        }
        if (metric == PMD_METRIC_REL) {
            num = sqrt(cta_sum(a, red));
            den = sqrt(cta_sum(b, red));
        } else {
            num = sqrt(cta_max(mx, red));   // max_i |dq_i| = sqrt(max_i |dq_i|^2)
        }
    }
    double delta = metric == PMD_METRIC_REL ? (den > 0 ? num / den : 0.0) : num;
    int n_stop = n_fin;
    bool list_ok = false;
    for (int nn = n_in; nn < n_fin; ++nn) {
        const long idx = nn - n_in;
        const double* Gp = Gwin ? Gwin + (size_t)idx * (nsteps + 1) * 3 * n : nullptr;
        double* co = cout + idx * S;
        double* cn = cur + (idx + 1) * S;
        const double* J = jumps ? jumps + idx * S : nullptr;
        const double* P = prev + (idx + 1) * S;
        // the jump and the previous iterate of the thread's own atom, loaded before the interval
        // so that they arrive during its force evaluations (one atom per thread: more would
        // not fit in registers, and those shapes read them after the interval)
        constexpr bool PRE = KMAX == 1;
        double Jo[KMAX][6], Po[KMAX][3];
#pragma unroll
        for (int k = 0; k < KMAX && PRE; ++k) {
            const int i = threadIdx.x + k * blockDim.x;
#pragma unroll
            for (int c = 0; c < 6; ++c) Jo[k][c] = (J && i < n) ? J[c * n + i] : 0.0;
#pragma unroll
            for (int al = 0; al < 3; ++al) Po[k][al] = i < n ? P[al * n + i] : 0.0;
        }
        coarse_interval_cta<real, KMAX>(s, own, n, box, pot, L, nsteps, (int64_t)nn, Gp, list_ok, status);
        // jump, writes and error sums on the owning thread of each atom (the force evaluation
        // ended with a CTA barrier, so no thread still reads q)
        double a = 0.0, b = 0.0, mx = 0.0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int i = threadIdx.x + k * blockDim.x;
            if (i < n) {
                if (!PRE) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) Jo[k][c] = J ? J[c * n + i] : 0.0;
#pragma unroll
                    for (int al = 0; al < 3; ++al) Po[k][al] = P[al * n + i];
                }
                double d2 = 0.0;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const double c = s.q[al * n + i];
                    co[al * n + i] = c;
                    const double u = J ? c + Jo[k][al] : c;
                    s.q[al * n + i] = u;
                    cn[al * n + i] = u;
                    if (!isfinite(u)) bad = true;
                    const double pp = Po[k][al];
                    d2 += (u - pp) * (u - pp);
                    b += pp * pp;
                }
                a += d2;
                mx = fmax(mx, d2);
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const double c = own.v[k][al];
                    co[3 * n + al * n + i] = c;
                    const double u = J ? c + Jo[k][3 + al] : c;
                    own.v[k][al] = u;
                    cn[3 * n + al * n + i] = u;
                    if (!isfinite(u)) bad = true;
                }
                s.qf[i] = wrap_f32(s.q[i], s.q[n + i], s.q[2 * n + i], box);
            }
        }
        const int anybad = __syncthreads_or(bad ? 1 : 0);
        if (metric == PMD_METRIC_REL) {
            num += sqrt(cta_sum(a, red));
            den += sqrt(cta_sum(b, red));
            delta = num / den;
        } else {
            num = fmax(num, sqrt(cta_max(mx, red)));
            delta = num;
        }
        if (anybad || !isfinite(delta)) delta = INFINITY;
        if (!(delta <= delta_expl)) {
            n_stop = nn;
            break;
        }
    }
    if (threadIdx.x == 0) {
        res->delta = delta;
        res->n_stop = n_stop;
    }
}

}  // namespace pmd

#include "sweep_cluster.cuh"

namespace pmd {

// G_{l,n} for every interval n of a window, l = 0..L, all atoms: [count][L+1][3][natoms]
__global__ void k_noise_window(uint64_t seed, int64_t n0, int count, int L1, int natoms, double* __restrict__ G) {
    const long total = (long)count * L1 * natoms;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
        const int i = (int)(x % natoms);
        const long t = x / natoms;
        const int ell = (int)(t % L1);
        const long c = t / L1;
        double g[3];
        normals3(seed, n0 + c, ell, i, g);
        double* out = G + ((c * L1 + ell) * 3) * natoms + i;
        out[0] = g[0];
        out[natoms] = g[1];
        out[2 * (long)natoms] = g[2];
    }
}

template <typename real, int KMAX, class CP>
struct SweepK {
    static auto ptr() { return &k_parareal_sweep<real, KMAX, CP>; }
};

int parareal_sweep(pmd_engine* e, int n_in, int n_fin, const double* jumps, const double* prev, double* cur,
                   double* cout, double delta_expl, int metric, int L, const pmd_langevin& lp, double* delta_host,
                   int* n_stop_host, cudaStream_t st) {
    const int n = e->p.natoms;
    int threads, kmax;
    coarse_shape(n, threads, kmax);
    threads = std::max(threads, 64);
    kmax = (n + threads - 1) / threads;
    const LangevinDev Ld = make_langevin(lp);
    const double* B = e->p.box;
    SweepResult* res = e->s_result.as<SweepResult>();
    // the window's Gaussian increments, drawn by the whole GPU ahead of the sequential sweep
    const int count = n_fin - n_in;
    double* Gwin = nullptr;
    if (count > 0 && L > 0) {
        const size_t need = (size_t)count * (L + 1) * 3 * n * sizeof(double);
        int rc0 = e->s_noise.ensure(need);
        if (rc0) return rc0;
        Gwin = e->s_noise.as<double>();
        const long total = (long)count * (L + 1) * n;
        const long blocks = std::min<long>((total + 255) / 256, (long)e->num_sms * 16);
        k_noise_window<<<(unsigned)blocks, 256, 0, st>>>(lp.seed, (int64_t)n_in, count, L + 1, n, Gwin);
        PMD_CUDA_TRY(cudaGetLastError());
    }
    auto go = [&](auto kern, auto cp, size_t sm) -> int {
        PMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<1, threads, sm, st>>>(n, B[0], B[1], B[2], cp, Ld, L, n_in, n_fin, jumps, prev, cur, cout, delta_expl,
                                     metric, Gwin, res, e->status.as<int>());
        PMD_CUDA_TRY(cudaGetLastError());
        return PMD_OK;
    };
    int rc;
    if (e->p.coarse_kind == PMD_COARSE_FS && n >= 64 && n <= EAM_LIST_MAX_ATOMS) {
        // the atoms of each interval spread over a cluster of up to 8 CTAs (SMs)
        const int K = std::min(SWEEP_CLUSTER_MAX, (n + 31) / 32), m = (n + K - 1) / K;
        // threads: S W per own atom in the pair passes, and three warps per 32 own atoms (the
        // axis split of the integrator); at most 512
        const int S = n <= 256 ? 2 : 1, rb = e->p.coarse.precision == PMD_FP64 ? 8 : 4;
        const int cthreads = std::max((S * sc_workers(rb) * m + 31) / 32 * 32, 96 * ((m + 31) / 32));
        const size_t csm = sweep_cluster_smem_bytes(n, m, K, S, rb);
        const FSDev fs = make_fs(e->p.coarse);
        auto kern = e->p.coarse.precision == PMD_FP64 ? k_parareal_sweep_cluster<double> : k_parareal_sweep_cluster<float>;
        PMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(K);
        cfg.blockDim = dim3(cthreads);
        cfg.dynamicSmemBytes = csm;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        PMD_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, n, m, B[0], B[1], B[2], fs, Ld, L, n_in, n_fin, jumps, prev, cur,
                                        cout, delta_expl, metric, (const double*)Gwin, res, e->status.as<int>()));
        rc = PMD_OK;
    } else {
        rc = coarse_dispatch<SweepK>(e, n, kmax, go);
    }
    if (rc) return rc;
    SweepResult* h = static_cast<SweepResult*>(e->pinned);
    PMD_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(SweepResult), cudaMemcpyDeviceToHost, st));
    PMD_CUDA_TRY(cudaStreamSynchronize(st));
    *delta_host = h->delta;
    *n_stop_host = h->n_stop;
    return PMD_OK;
}

// ---- jumps ------------------------------------------------------------------------------------
__global__ void k_jumps(const double* __restrict__ f, const double* __restrict__ c, double* __restrict__ j, long count) {
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < count; x += (long)gridDim.x * blockDim.x)
        j[x] = f[x] - c[x];
}

int jumps_launch(long count, const double* f, const double* c, double* j, int num_sms, cudaStream_t st) {
    if (count <= 0) return PMD_OK;
    const long blocks = std::min<long>((count + 255) / 256, (long)num_sms * 8);
    k_jumps<<<(unsigned)blocks, 256, 0, st>>>(f, c, j, count);
    PMD_CUDA_TRY(cudaGetLastError());
    return PMD_OK;
}

}  // namespace pmd
