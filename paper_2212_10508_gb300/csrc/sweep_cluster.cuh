// Parareal correction sweep (Algorithm 2's inner loop) on a thread-block cluster of K <= 8 CTAs,
// for the Finnis-Sinclair coarse potential: cur_{n+1} = C(cur_n) + J_n for n = N_init ..., with
// the running slab error and the explosion test.
//
// The sweep is sequential in n; what a cluster adds is the atoms of each interval spread over K
// SMs (the one-CTA sweep runs every FP64 integrator operation, the EAM pair passes and the error
// sums of all atoms on one SM).  CTA r owns the atoms [r m, r m + m), m = ceil(n / K), and keeps
// a full copy of the wrapped FP32 positions (and, in FP64 mode, of the FP64 rows) and of the
// embedding derivatives F'(rho) in its own shared memory; the owner of an atom writes its new
// values into every CTA's copy through distributed shared memory (plain stores), followed by a
// cluster barrier.  The positions are double-buffered: a publication goes to the buffer nobody
// reads until the barrier after it, so a CTA still in its force pass never sees a half-updated
// copy (F'(rho) needs no second buffer: a position barrier always separates two force
// evaluations).  Per interval of one step: the corrected state, the error partial sums and the
// list staleness of the previous interval, the F'(rho) of each of the two force evaluations, and
// the drifted positions -- four cluster barriers.  Every decision (rebuilding the Verlet lists,
// stopping at an explosion) is taken from values every CTA combines in the same order, so all
// CTAs take the same branches and reach the same barriers.
//
// Each atom's arithmetic is that of the one-CTA coarse kernels: the same Verlet list (every pair
// within max(d, c) + skin, rebuilt for all atoms when any atom has moved more than half the skin),
// split into the same S sub-lists by neighbour index, the same pair terms summed in the same order,
// the same integrator steps -- so C(cur_n) equals, bit for bit, the C(prev_n) that k_coarse_batch
// computes for the jumps.  Only the slab error's sum over atoms runs in another order (per CTA,
// then over the CTAs in rank order).  The thread layout differs from the one-CTA kernels: W
// workers per sub-list in the pair passes, and the FP64 integrator split by axis (see the kernel).
#pragma once

#include <cfloat>

#include <cooperative_groups.h>

#include "eam_device.cuh"
#include "langevin_device.cuh"

namespace pmd {

constexpr int SWEEP_CLUSTER_MAX = 8;   // portable cluster size
// Worker threads per sub-list in the pair passes and the list build: 8 in FP32-bulk mode, 4 in
// FP64 mode (whose pair geometry is FP64: more warps only queue on the FP64 units).
__host__ __device__ constexpr int sc_workers(int real_bytes) { return real_bytes == 4 ? 8 : 4; }

// Per-entry terms of the pair passes: the density pass's workers store the pair geometry
// (r, r_j - r_i), r = +inf for an entry outside the screen radius; the force pass's workers
// replace it with (g, r_j - r_i), zeros for an entry with no force term.
template <typename real>
struct alignas(4 * sizeof(real)) ScTerm {
    real x, y, z, w;
};

struct SweepClusterShared {
    double* qb0;           // [3][n] positions, two buffers (all atoms' in FP64 mode, the own atoms'
    double* qb1;           // in FP32 mode; named, not an array indexed at run time, which would
                           // put the pointers in local memory)
    float4* qfb0;          // [n] wrapped FP32 positions (replicated, two buffers)
    float4* qfb1;
    double* q;             // the current buffers
    float4* qf;
    double* dF;            // [n] F'(rho) of all atoms (replicated; FP64 mode)
    float* dFf;            // [n] the same in FP32 mode (the FP32 values themselves)
    double* F;             // [3][m] forces of the own atoms
    float4* qref;          // [m] own atoms' wrapped positions at the last list build
    double* part;          // [K][4] per-CTA partial sums (|dq|^2, |q_prev|^2, max |dq_i|^2, non-finite)
    int* stale;            // [K] per-CTA list staleness
    unsigned short* nbl;   // own atoms' Verlet lists, eam_pidx layout over m atoms
    unsigned char* nbc;    // [S][m] sub-list lengths (eam_build_list's parity split)
    void* term;            // [m][S][EAM_LIST_CAP / S + 1] ScTerm<real>: pair terms of each sub-list
    double* stg;           // [6][m] own atoms' per-axis values staged for the per-atom steps
    float* stgf;           // [3][m] own atoms' wrapped FP32 coordinates, staged
};

// Entries per sub-list in the term array (one of padding, so that the sub-lists of a warp start in
// different banks).
__host__ __device__ inline int sc_term_pitch(int S) { return EAM_LIST_CAP / S + 1; }

__host__ __device__ inline size_t sweep_cluster_smem_bytes(int n, int m, int K, int S, int real_bytes) {
    size_t b = (size_t)n * (2 * 3 * 8 + 8) + 32;   // two q buffers, dF
    b += (size_t)n * 2 * 16 + 32;                 // two qf buffers
    b += (size_t)m * 3 * 8 + (size_t)m * 16 + 16;
    b += (size_t)K * 4 * 8 + (size_t)K * 4 + 16;
    b += (size_t)m * EAM_LIST_CAP * 2 + 2 * m;
    b += (size_t)m * S * sc_term_pitch(S) * 4 * real_bytes;
    b += (size_t)n * 4 + (size_t)m * 6 * 8 + (size_t)m * 3 * 4;   // dFf, stg, stgf
    b += 16 * 16 + 32;   // alignment of the fifteen carved arrays (16 bytes; the terms 32)
    return (b + 15) / 16 * 16;
}

__device__ inline SweepClusterShared sweep_cluster_carve(unsigned char* smem, int n, int m, int K, int S,
                                                        int real_bytes) {
    SweepClusterShared s;
    size_t o = 0;
    auto take = [&](size_t bytes, size_t align) {
        o = (o + align - 1) / align * align;
        unsigned char* p = smem + o;
        o += bytes;
        return p;
    };
    s.qb0 = reinterpret_cast<double*>(take((size_t)3 * n * 8, 16));
    s.qb1 = reinterpret_cast<double*>(take((size_t)3 * n * 8, 16));
    s.dF = reinterpret_cast<double*>(take((size_t)n * 8, 16));
    s.qfb0 = reinterpret_cast<float4*>(take((size_t)n * 16, 16));
    s.qfb1 = reinterpret_cast<float4*>(take((size_t)n * 16, 16));
    s.q = s.qb0;
    s.qf = s.qfb0;
    s.F = reinterpret_cast<double*>(take((size_t)3 * m * 8, 16));
    s.qref = reinterpret_cast<float4*>(take((size_t)m * 16, 16));
    s.part = reinterpret_cast<double*>(take((size_t)K * 4 * 8, 16));
    s.stale = reinterpret_cast<int*>(take((size_t)K * 4, 16));
    s.nbl = reinterpret_cast<unsigned short*>(take((size_t)m * EAM_LIST_CAP * 2, 16));
    s.nbc = reinterpret_cast<unsigned char*>(take((size_t)2 * m, 16));
    s.term = take((size_t)m * S * sc_term_pitch(S) * 4 * real_bytes, 32);
    s.dFf = reinterpret_cast<float*>(take((size_t)n * 4, 16));
    s.stg = reinterpret_cast<double*>(take((size_t)m * 6 * 8, 16));
    s.stgf = reinterpret_cast<float*>(take((size_t)m * 3 * 4, 16));
    return s;
}

// The cluster's view: rank, owned atoms, the S sub-lists of an atom (the one-CTA kernels' split of
// its pairs) and the T = S W threads of an atom in the pair passes: thread t of the CTA works for
// own atom t / T, sub-list (t / W) mod S, as worker t mod W.
struct SweepOwn {
    int K, rank, a0, mown, m, S, W, T;
};

// Own atoms' Verlet lists: the sub-lists of eam_build_list (sub-list u of an atom holds the pairs
// within the reach with neighbour index j = u mod S, in index order) over the m own slots.  The
// W workers of a sub-list scan consecutive chunks of its candidates j, count their hits, take
// their offsets from a prefix sum over the workers (shuffles) and write their hits in a second
// scan, so the sub-list comes out in index order.
__device__ __forceinline__ void sc_build_lists(const SweepClusterShared& s, const SweepOwn& w, int n, const double box[3],
                                      float reach2, int* status) {
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const int S = w.S, cap = EAM_LIST_CAP / S;
    const int span = (w.T * w.m + 31) / 32 * 32;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {   // whole warps: the shuffles take every lane
        const int li = t / w.T, u = (t / w.W) % S, v = t % w.W, i = w.a0 + li;
        const bool act = li < w.mown;
        const int ncls = act ? (n - u + S - 1) / S : 0;   // candidates j = u + S c, c < ncls
        const int per = (ncls + w.W - 1) / w.W;
        const int c0 = v * per, c1 = c0 + per < ncls ? c0 + per : ncls;
        const float4 qi = act ? s.qf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int hits = 0;
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const int j = u + S * c;
            hits += j != i && r2_f32(mi_f32(qi, s.qf[j], boxf, ibf)) < reach2;
        }
        int incl = hits;   // inclusive prefix over the workers of this sub-list
        for (int d = 1; d < w.W; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d, w.W);
            if (v >= d) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, w.W - 1, w.W);
        int k = incl - hits;
        for (int c = c0; c < c1 && k < cap; ++c) {
            const int j = u + S * c;
            if (j == i || !(r2_f32(mi_f32(qi, s.qf[j], boxf, ibf)) < reach2)) continue;
            s.nbl[eam_pidx(li, k * S + u, w.m, S)] = (unsigned short)j;
            ++k;
        }
        if (act && v == 0) {
            if (total > cap) flag(status, ST_NEIGH);
            s.nbc[u * w.m + li] = (unsigned char)(total > cap ? cap : total);
            if (u == 0) s.qref[li] = qi;
        }
    }
}

// The two EAM pair passes of the own atoms, with the sums of the one-CTA kernels (eam_forces_cta):
// per sub-list, the terms of its entries added in entry order, then the S sub-lists' sums combined
// by an xor-shuffle.  The W workers of a sub-list take entries v, v + W, ...: in the density
// pass they store each entry's pair geometry in the term array (the force pass reuses it, as the
// one-CTA kernels' pair cache does, with the same bits); in the force pass they compute g from it
// and F'(rho_j).  After a warp barrier the sub-list's first worker adds the terms in order with
// the one-CTA loops' operations (an entry with no term adds exact zeros), so the sums have their
// bits.  The F'(rho) of the own atoms go to every CTA before the force pass.  All threads; ends
// with a CTA barrier.
template <typename real>
__device__ __forceinline__ void sc_forces(const SweepClusterShared& s, const SweepOwn& w, int n, const double box[3], const FSDev& p,
                          cooperative_groups::cluster_group& cl) {
    EamShared e{};
    e.q = s.q;
    e.qf = s.qf;
    e.dF = s.dF;
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const real d_ = (real)p.d, c_ = (real)p.c, c0 = (real)p.c0, c1 = (real)p.c1, c2 = (real)p.c2;
    const int S = w.S, pitch = sc_term_pitch(S);
    const int span = (w.T * w.m + 31) / 32 * 32;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const int li = t / w.T, u = (t / w.W) % S, v = t % w.W, i = w.a0 + li;
        const bool act = li < w.mown;
        const int cnt = act ? s.nbc[u * w.m + li] : 0;
        ScTerm<real>* tr = reinterpret_cast<ScTerm<real>*>(s.term) + (size_t)(li * S + u) * pitch;
        const float4 qi = act ? s.qf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
        for (int k = v; k < cnt; k += w.W) {
            const int j = s.nbl[eam_pidx(li, k * S + u, w.m, S)];
            real dv[3], r;
            ScTerm<real> y{real(INFINITY), 0, 0, 0};
            if (pair_in<real>(e, n, i, j, qi, box, boxf, ibf, p.screen2, r, dv)) y = ScTerm<real>{r, dv[0], dv[1], dv[2]};
            tr[k] = y;
        }
        __syncwarp();
        real rho = 0;
        if (v == 0)
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const real r = tr[k].x;
                const real x = r < d_ ? r - d_ : real(0);
                rho += x * x;
            }
        if (S == 2) rho += __shfl_xor_sync(0xffffffffu, rho, w.W);
        if (act && u == 0 && v == 0) {
            if constexpr (sizeof(real) == 4) {   // the value the one-CTA kernels store as a double
                const float dF = rho > 0.f ? -0.5f * (float)p.A / sqrtf(rho) : 0.0f;
                for (int r2 = 0; r2 < w.K; ++r2) cl.map_shared_rank(s.dFf, r2)[i] = dF;
            } else {
                const double dF = (double)rho > 0.0 ? -p.A / (2.0 * sqrt((double)rho)) : 0.0;
                for (int r2 = 0; r2 < w.K; ++r2) cl.map_shared_rank(s.dF, r2)[i] = dF;
            }
        }
    }
    cl.sync();   // every CTA has every F'(rho); the density terms are read
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const int li = t / w.T, u = (t / w.W) % S, v = t % w.W, i = w.a0 + li;
        const bool act = li < w.mown;
        const int cnt = act ? s.nbc[u * w.m + li] : 0;
        ScTerm<real>* tr = reinterpret_cast<ScTerm<real>*>(s.term) + (size_t)(li * S + u) * pitch;
        const real* dFr;
        if constexpr (sizeof(real) == 4) dFr = s.dFf;
        else dFr = s.dF;
        const real dFi = act ? dFr[i] : real(0);
#pragma unroll 2
        for (int k = v; k < cnt; k += w.W) {
            const int j = s.nbl[eam_pidx(li, k * S + u, w.m, S)];
            const ScTerm<real> gm = tr[k];
            real g;
            ScTerm<real> y{0, 0, 0, 0};
            if (gm.x < real(INFINITY) && eam_pair_g<real>(gm.x, dFi, dFr[j], d_, c_, c0, c1, c2, g))
                y = ScTerm<real>{g, gm.y, gm.z, gm.w};
            tr[k] = y;
        }
        __syncwarp();
        real f0 = 0, f1 = 0, f2 = 0;
        if (v == 0)
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const ScTerm<real> y = tr[k];
                f0 += y.x * y.y;
                f1 += y.x * y.z;
                f2 += y.x * y.w;
            }
        if (S == 2) {
            f0 += __shfl_xor_sync(0xffffffffu, f0, w.W);
            f1 += __shfl_xor_sync(0xffffffffu, f1, w.W);
            f2 += __shfl_xor_sync(0xffffffffu, f2, w.W);
        }
        if (act && u == 0 && v == 0) {
            s.F[li] = (double)f0;
            s.F[w.m + li] = (double)f1;
            s.F[2 * w.m + li] = (double)f2;
        }
    }
    __syncthreads();
}

// Coordinate al of own atom i into the other position buffer (nb: its index), which becomes the
// current one after the next cluster barrier: to every CTA in FP64 mode (its pair geometry reads
// the FP64 rows), to the own CTA only in FP32 mode (the pair passes read only the FP32 copy; the
// integrator, the jumps and the error sums only own atoms).
template <typename real>
__device__ __forceinline__ void sc_publish_row(const SweepClusterShared& s, const SweepOwn& w, int n, int nb, int al,
                                               int i, double x, cooperative_groups::cluster_group& cl) {
    double* q = nb ? s.qb1 : s.qb0;
    if constexpr (sizeof(real) == 4) {
        q[al * n + i] = x;
    } else {
        for (int r = 0; r < w.K; ++r) cl.map_shared_rank(q, r)[al * n + i] = x;
    }
}

// Own atom ow's wrapped FP32 position, from its three staged coordinates, into every CTA's other
// FP32 buffer; returns 1 if the atom moved more than half the skin since the last list build.
__device__ __forceinline__ int sc_publish_qf(const SweepClusterShared& s, const SweepOwn& w, int nb, int ow, int i,
                                             const float boxf[3], const float ibf[3], float lim2,
                                             cooperative_groups::cluster_group& cl) {
    const float4 qw = make_float4(s.stgf[ow], s.stgf[w.m + ow], s.stgf[2 * w.m + ow], 0.f);
    float4* qf = nb ? s.qfb1 : s.qfb0;
    for (int r = 0; r < w.K; ++r) cl.map_shared_rank(qf, r)[i] = qw;
    return r2_f32(mi_f32(s.qref[ow], qw, boxf, ibf)) > lim2;
}

// Gaussian increment of coordinate al of atom i at sub-step ell (coarse_noise's values).
__device__ __forceinline__ double sc_noise1(const LangevinDev& L, const double* Gpre, int64_t nid, int ell, int i,
                                            int n, int al) {
    if (Gpre) return Gpre[((size_t)ell * 3 + al) * n + i];
    double G[3];
    normals3(L.seed, nid, ell, i, G);
    return al == 0 ? G[0] : (al == 1 ? G[1] : G[2]);
}

// Switch to the buffers published into (after the cluster barrier that follows the publication).
__device__ __forceinline__ void sc_flip(SweepClusterShared& s, int& cb) {
    cb ^= 1;
    s.q = cb ? s.qb1 : s.qb0;
    s.qf = cb ? s.qfb1 : s.qfb0;
}

// Staleness of the own atoms to every CTA (called by every thread; thread 0 writes).
__device__ __forceinline__ void sc_publish_stale(const SweepClusterShared& s, const SweepOwn& w, int st,
                                                 cooperative_groups::cluster_group& cl) {
    const int any = __syncthreads_or(st);
    if (threadIdx.x == 0)
        for (int r = 0; r < w.K; ++r) cl.map_shared_rank(s.stale, r)[w.rank] = any;
}

// After the cluster barrier that follows sc_publish_stale: rebuild the own lists if any CTA's atoms
// moved (every CTA sees the same flags, so all rebuild together).  Ends with a CTA barrier.
__device__ __forceinline__ void sc_refresh(const SweepClusterShared& s, const SweepOwn& w, int n, const double box[3],
                                           const FSDev& p, int* status) {
    int any = 0;
    for (int r = 0; r < w.K; ++r) any |= s.stale[r];
    if (any) {
        const float reach = sqrtf(p.screen2) + EAM_SKIN;
        sc_build_lists(s, w, n, box, reach * reach, status);
    }
    __syncthreads();
}

// The per-atom error terms into thread 0: for the relative metric the sums of a = |dq_i|^2 and
// b = |q_i^prev|^2 (FP64), for the maximum metric the maximum of |dq_i|^2 as the bits of a
// non-negative double (integer maxima order them as the values, with no FP64 instruction).  The
// atoms sit on the lanes of warps 3 ob, ob < nb; xor-butterflies within those warps, then their
// results in order (a CTA barrier when nb > 1; nb is the same for every thread).
__device__ __forceinline__ void sc_atom_reduce(int nb, int metric, double a, double b, unsigned long long mx,
                                               double* red, double& A, double& B, unsigned long long& M) {
    const int wv = threadIdx.x >> 5, ob = wv / 3;
    if (wv % 3 == 0 && ob < nb) {
        for (int o = 16; o > 0; o >>= 1) {
            if (metric == PMD_METRIC_REL) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
            } else {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
                mx = y > mx ? y : mx;
            }
        }
        if ((threadIdx.x & 31) == 0 && ob > 0) {
            red[3 * ob] = a;
            red[3 * ob + 1] = b;
            red[3 * ob + 2] = __longlong_as_double((long long)mx);
        }
    }
    if (nb > 1) __syncthreads();
    if (threadIdx.x == 0) {
        A = a;
        B = b;
        M = mx;
        for (int k = 1; k < nb; ++k) {
            if (metric == PMD_METRIC_REL) {
                A += red[3 * k];
                B += red[3 * k + 1];
            } else {
                const unsigned long long y = (unsigned long long)__double_as_longlong(red[3 * k + 2]);
                M = y > M ? y : M;
            }
        }
    }
}

// The largest x >= 0 with sqrt(x) <= e (e finite, >= 0), as bits: sqrt is correctly rounded and
// monotonic, so sqrt(y) <= e exactly when y <= x, and the maximum metric's explosion test needs no
// square root per interval.  Starts from e * e and steps by ulps (a few steps at most; bounded).
__device__ inline unsigned long long sc_sq_threshold(double e) {
    double x = e * e;
    if (isinf(x)) x = DBL_MAX;
    for (int k = 0; k < 64 && x > 0.0 && sqrt(x) > e; ++k) x = nextafter(x, 0.0);
    for (int k = 0; k < 64 && x < DBL_MAX && sqrt(nextafter(x, INFINITY)) <= e; ++k) x = nextafter(x, INFINITY);
    return (unsigned long long)__double_as_longlong(x);
}

// Every CTA's partial sums (after the cluster barrier) combined in rank order: (a, b, mx, bad).
__device__ __forceinline__ void sc_totals(const SweepClusterShared& s, const SweepOwn& w, int metric, double& a,
                                          double& b, unsigned long long& mx, int& bad) {
    a = 0.0;
    b = 0.0;
    mx = 0;
    bad = 0;
    for (int r = 0; r < w.K; ++r) {
        if (metric == PMD_METRIC_REL) {
            a += s.part[4 * r];
            b += s.part[4 * r + 1];
        } else {
            const unsigned long long y = (unsigned long long)__double_as_longlong(s.part[4 * r + 2]);
            mx = y > mx ? y : mx;
        }
        bad |= s.part[4 * r + 3] != 0.0;
    }
}

template <typename real>
__global__ void __launch_bounds__(512, 1) k_parareal_sweep_cluster(
    int n, int m, double b0, double b1, double b2, FSDev fs, LangevinDev L, int nsteps, int n_in, int n_fin,
    const double* __restrict__ jumps, const double* __restrict__ prev, double* __restrict__ cur,
    double* __restrict__ cout, double delta_expl, int metric, const double* __restrict__ Gwin, SweepResult* res,
    int* status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[33];   // CTA reductions (cta_sum's 33 doubles, or 3 per warp)
    __shared__ int s_stop;       // the explosion test's outcome, from thread 0
    SweepOwn w;
    w.K = (int)cl.num_blocks();
    w.rank = (int)cl.block_rank();
    w.m = m;
    w.a0 = w.rank * m;
    w.mown = w.a0 >= n ? 0 : (n - w.a0 < m ? n - w.a0 : m);
    w.S = n <= 256 ? 2 : 1;   // the entry split of the one-CTA kernels' launch shape
    w.W = sc_workers((int)sizeof(real));
    w.T = w.S * w.W;
    SweepClusterShared s = sweep_cluster_carve(smem, n, m, w.K, w.S, (int)sizeof(real));
    int cb = 0;   // current position buffer (the same in every CTA: all publish at the same points)
    const double box[3] = {b0, b1, b2};
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const float lim2 = 0.25f * EAM_SKIN * EAM_SKIN;
    const long SS = 6L * n;
    const int t = threadIdx.x, wv = t >> 5;
    // Axis thread (al, ow): coordinate al of own atom ow, on lane ow mod 32 of warp 3 (ow / 32) + al.
    // An FP64 instruction holds its SM sub-partition's FP64 unit for the same time whatever the
    // number of active lanes, so the integrator's and the jumps' FP64 arithmetic is split by axis
    // over three warps (three sub-partitions).  The al = 0 threads also take the per-atom steps
    // (the FP32 position copy, the list staleness, the error terms) from staged values.
    const int nb = (m + 31) >> 5;
    const int al = wv % 3, ow = (wv / 3) * 32 + (t & 31);
    const bool mine = wv < 3 * nb && ow < w.mown;
    const bool atom = mine && al == 0;
    const int i = w.a0 + ow;
    const double Lb = al == 0 ? b0 : (al == 1 ? b1 : b2), iLb = 1.0 / Lb;
    // the window's first state: every CTA loads all positions, the axis threads their velocities
    for (int x = t; x < 3 * n; x += blockDim.x) s.q[x] = cur[x];
    double v = 0.0, vh = 0.0;
    if (mine) v = cur[3 * n + al * n + i];
    __syncthreads();
    for (int x = t; x < n; x += blockDim.x) s.qf[x] = wrap_f32(s.q[x], s.q[n + x], s.q[2 * n + x], box);
    __syncthreads();
    // error sums from n = n_in: |q^cur - q^prev| and |q^prev| of the first state
    {
        double a = 0.0, bb = 0.0, mx = 0.0;
        if (atom) {
            double d2 = 0.0;
            for (int c3 = 0; c3 < 3; ++c3) {
                const double c = cur[c3 * n + i], pp = prev[c3 * n + i];
                d2 += (c - pp) * (c - pp);
                bb += pp * pp;
            }
            a = d2;
            mx = d2;
        }
        const double A = cta_sum(a, red), B = cta_sum(bb, red), M = cta_max(mx, red);
        if (t == 0)
            for (int r = 0; r < w.K; ++r) {
                double* pr = cl.map_shared_rank(s.part, r) + 4 * w.rank;
                pr[0] = A;
                pr[1] = B;
                pr[2] = M;
                pr[3] = 0.0;
            }
    }
    sc_build_lists(s, w, n, box, (sqrtf(fs.screen2) + EAM_SKIN) * (sqrtf(fs.screen2) + EAM_SKIN), status);
    cl.sync();
    // The running error (thread 0).  Relative metric: num, den and delta as in Algorithm 2.  Maximum
    // metric: num2 = the running maximum of |dq_i|^2 as bits (NaN maxima are skipped, as fmax skips
    // them), delta = sqrt(num2), and the explosion test compares num2 with thr2.
    const unsigned long long INF_BITS = 0x7ff0000000000000ull;
    const bool e_inf = isinf(delta_expl) && delta_expl > 0.0;   // nothing explodes
    const bool e_neg = !(delta_expl >= 0.0);                     // everything explodes
    double num = 0.0, den = 0.0, delta = 0.0;
    unsigned long long num2 = 0, thr2 = 0;
    bool last_bad = false;
    if (t == 0) {
        double A, B;
        unsigned long long Mb;
        int bad;
        sc_totals(s, w, metric, A, B, Mb, bad);
        if (metric == PMD_METRIC_REL) {
            num = sqrt(A);
            den = sqrt(B);
            delta = den > 0 ? num / den : 0.0;
        } else {
            num2 = Mb;
            if (!e_inf && !e_neg) thr2 = sc_sq_threshold(delta_expl);
        }
    }
    int n_stop = n_fin;
    for (int nn = n_in; nn < n_fin; ++nn) {
        const long idx = nn - n_in;
        const double* Gp = Gwin ? Gwin + (size_t)idx * (nsteps + 1) * 3 * n : nullptr;
        double* co = cout + idx * SS;
        double* cn = cur + (idx + 1) * SS;
        const double* J = jumps ? jumps + idx * SS : nullptr;
        const double* P = prev + (idx + 1) * SS;
        double Jq = 0.0, Jv = 0.0, Pq = 0.0;
        if (mine) {
            if (J) {
                Jq = J[al * n + i];
                Jv = J[3 * n + al * n + i];
            }
            Pq = P[al * n + i];
        }
        // ---- C(cur_n): nsteps sub-steps of interval nn (coarse_interval_cta's arithmetic, per axis)
        bool bad = false;
        if (nsteps > 0) {
            double g = 0.0;
            if (mine) g = sc_noise1(L, Gp, (int64_t)nn, 0, i, n, al);
            sc_forces<real>(s, w, n, box, fs, cl);
            if (L.scheme == PMD_SCHEME_PAPER) vh = v;
            for (int ell = 0; ell < nsteps; ++ell) {
                const double s0 = sched_sigma(L, ell), s1 = sched_sigma(L, ell + 1);
                if (mine) {
                    const double F = s.F[al * m + ow];
                    const double q0 = s.q[al * n + i];
                    double qn;
                    if (L.scheme == PMD_SCHEME_PAPER) {
                        vh = half_kick(L, v, F, vh, s0, g);
                        qn = drift(q0, L.dt, vh);
                    } else {
                        double vv = kick_b(L, v, F);
                        qn = __dadd_rn(q0, __dmul_rn(L.hdt, vv));
                        vv = ou_o(L, vv, g);
                        qn = __dadd_rn(qn, __dmul_rn(L.hdt, vv));
                        v = vv;
                    }
                    if (!isfinite(qn)) bad = true;
                    if (fabs(qn - q0) > 0.5 * Lb) flag(status, ST_LOSTATOM);
                    sc_publish_row<real>(s, w, n, cb ^ 1, al, i, qn, cl);
                    s.stgf[al * m + ow] = wrap1_f32(qn, Lb, iLb);
                    if (L.scheme == PMD_SCHEME_PAPER || ell + 1 < nsteps) g = sc_noise1(L, Gp, (int64_t)nn, ell + 1, i, n, al);
                }
                __syncthreads();   // the three coordinates of every own atom are staged
                const int st = atom ? sc_publish_qf(s, w, cb ^ 1, ow, i, boxf, ibf, lim2, cl) : 0;
                sc_publish_stale(s, w, st, cl);
                cl.sync();   // positions and staleness of every atom
                sc_flip(s, cb);
                sc_refresh(s, w, n, box, fs, status);
                sc_forces<real>(s, w, n, box, fs, cl);
                if (mine) {
                    const double F = s.F[al * m + ow];
                    if (L.scheme == PMD_SCHEME_PAPER) v = half_kick(L, vh, F, vh, s1, g);
                    else v = kick_b(L, v, F);
                }
            }
        }
        if (bad) flag(status, ST_NONFINITE);
        // ---- jump, writes, error terms, and the corrected state to every CTA
        // (the outputs C(cur_n) and cur_{n+1} go to global memory after the cluster barrier below,
        // whose release would otherwise wait for those stores)
        int nonfin = bad ? 1 : 0;
        double oq = 0.0, ov = 0.0, uq = 0.0;
        if (mine) {
            oq = s.q[al * n + i];
            uq = J ? oq + Jq : oq;
            if (!isfinite(uq)) nonfin = 1;
            s.stg[al * m + ow] = uq - Pq;
            s.stg[(3 + al) * m + ow] = Pq;
            ov = v;
            v = J ? ov + Jv : ov;
            if (!isfinite(v)) nonfin = 1;
            sc_publish_row<real>(s, w, n, cb ^ 1, al, i, uq, cl);
            s.stgf[al * m + ow] = wrap1_f32(uq, Lb, iLb);
        }
        const int anybad = __syncthreads_or(nonfin);   // and the staged values are visible
        double a = 0.0, bb = 0.0;
        unsigned long long mxb = 0;
        int st = 0;
        if (atom) {
            double d2 = 0.0;
            for (int c3 = 0; c3 < 3; ++c3) {
                const double du = s.stg[c3 * m + ow];
                d2 += du * du;
            }
            if (metric == PMD_METRIC_REL) {
                a = d2;
                for (int c3 = 0; c3 < 3; ++c3) {
                    const double pp = s.stg[(3 + c3) * m + ow];
                    bb += pp * pp;
                }
            } else {
                mxb = (unsigned long long)__double_as_longlong(d2);
            }
            st = sc_publish_qf(s, w, cb ^ 1, ow, i, boxf, ibf, lim2, cl);
        }
        double A = 0.0, B = 0.0;
        unsigned long long Mb = 0;
        sc_atom_reduce(w.mown > 32 ? 2 : 1, metric, a, bb, mxb, red, A, B, Mb);
        if (t == 0)
            for (int r = 0; r < w.K; ++r) {
                double* pr = cl.map_shared_rank(s.part, r) + 4 * w.rank;
                pr[0] = A;
                pr[1] = B;
                pr[2] = __longlong_as_double((long long)Mb);
                pr[3] = anybad ? 1.0 : 0.0;
            }
        sc_publish_stale(s, w, st, cl);
        cl.sync();   // corrected state, partial sums and staleness of every CTA
        if (mine) {
            co[al * n + i] = oq;
            cn[al * n + i] = uq;
            co[3 * n + al * n + i] = ov;
            cn[3 * n + al * n + i] = v;
        }
        sc_flip(s, cb);
        if (t == 0) {   // the running error and the explosion test in one thread
            double TA, TB;
            unsigned long long TM;
            int tbad;
            sc_totals(s, w, metric, TA, TB, TM, tbad);
            if (metric == PMD_METRIC_REL) {
                num += sqrt(TA);
                den += sqrt(TB);
                delta = num / den;
                if (tbad || !isfinite(delta)) delta = INFINITY;
                s_stop = !(delta <= delta_expl);
            } else {
                if (TM <= INF_BITS) num2 = (num2 > INF_BITS || TM > num2) ? TM : num2;
                last_bad = tbad || num2 >= INF_BITS;   // delta = INFINITY
                s_stop = e_inf ? 0 : (e_neg || last_bad || num2 > thr2);
            }
        }
        __syncthreads();
        if (s_stop) {
            n_stop = nn;
            break;
        }
        sc_refresh(s, w, n, box, fs, status);
    }
    if (w.rank == 0 && t == 0) {
        if (metric != PMD_METRIC_REL) delta = last_bad ? INFINITY : sqrt(__longlong_as_double((long long)num2));
        res->delta = delta;
        res->n_stop = n_stop;
    }
    cl.sync();   // no CTA leaves while another may still write into its shared memory
}

}  // namespace pmd
