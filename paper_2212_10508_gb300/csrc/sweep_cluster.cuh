// Parareal correction sweep (Algorithm 2's inner loop) on a thread-block cluster of K <= 8 CTAs,
// for the Finnis-Sinclair coarse potential: cur_{n+1} = C(cur_n) + J_n for n = N_init ..., with
// the running slab error and the explosion test.
//
// The sweep is sequential in n; what a cluster adds is the atoms of each interval spread over K
// SMs (the one-CTA sweep runs every FP64 integrator operation, the EAM pair passes and the error
// sums of all atoms on one SM).  CTA r owns the atoms [r m, r m + m), m = ceil(n / K), and keeps
// a full copy of the positions (FP64 rows and the wrapped FP32 copy) and of the embedding
// derivatives F'(rho) in its own shared memory; the owner of an atom writes its new values into
// every CTA's copy through distributed shared memory (plain stores), followed by a cluster
// barrier.  The positions are double-buffered: a publication goes to the buffer nobody reads
// until the barrier after it, so a CTA still in its force pass never sees a half-updated copy
// // (F'(rho) needs no second buffer: a position barrier always separates two force evaluations).
// Per interval of one step: the corrected state and the list staleness of the previous interval,
// the F'(rho) of each of the two force evaluations, and the drifted positions -- four cluster
// barriers.  Every decision (rebuilding the Verlet lists, stopping at
// an explosion) is taken from values every CTA combines in the same order, so all CTAs take the
// same branches and reach the same barriers.
//
// Each atom's arithmetic is that of the one-CTA coarse kernels: the same Verlet list (every pair
// within max(d, c) + skin in index order, rebuilt for all atoms when any atom has moved more than
// half the skin), the same split of the pair entries over S threads per atom, the same pair
// terms and integrator steps -- so C(cur_n) equals, bit for bit, the C(prev_n) that
// k_coarse_batch computes for the jumps.  Only the slab error's sum over atoms runs in another
// order (per CTA, then over the CTAs in rank order).
#pragma once

#include <cooperative_groups.h>

#include "eam_device.cuh"
#include "langevin_device.cuh"

namespace pmd {

constexpr int SWEEP_CLUSTER_MAX = 8;   // portable cluster size

struct SweepClusterShared {
    double* qb[2];         // [3][n] all positions (replicated, two buffers)
    float4* qfb[2];        // [n] wrapped FP32 positions (replicated, two buffers)
    double* q;             // the current buffers
    float4* qf;
    double* dF;            // [n] F'(rho) of all atoms (replicated)
    double* F;             // [3][m] forces of the own atoms
    float4* qref;          // [m] own atoms' wrapped positions at the last list build
    double* part;          // [K][4] per-CTA partial sums (|dq|^2, |q_prev|^2, max |dq_i|^2, non-finite)
    int* stale;            // [K] per-CTA list staleness
    unsigned short* nbl;   // own atoms' Verlet lists, eam_pidx layout over m atoms
    unsigned char* nbc;    // [S][m] sub-list lengths (eam_build_list's parity split)
};

__host__ __device__ inline size_t sweep_cluster_smem_bytes(int n, int m, int K) {
    size_t b = (size_t)n * (2 * 3 * 8 + 8) + 32;   // two q buffers, dF
    b += (size_t)n * 2 * 16 + 32;                 // two qf buffers
    b += (size_t)m * 3 * 8 + (size_t)m * 16 + 16;
    b += (size_t)K * 4 * 8 + (size_t)K * 4 + 16;
    b += (size_t)m * EAM_LIST_CAP * 2 + 2 * m;
    b += 16 * 16;   // alignment of the eleven carved arrays to 16 bytes
    return (b + 15) / 16 * 16;
}

__device__ inline SweepClusterShared sweep_cluster_carve(unsigned char* smem, int n, int m, int K) {
    SweepClusterShared s;
    size_t o = 0;
    auto take = [&](size_t bytes, size_t align) {
        o = (o + align - 1) / align * align;
        unsigned char* p = smem + o;
        o += bytes;
        return p;
    };
    s.qb[0] = reinterpret_cast<double*>(take((size_t)3 * n * 8, 16));
    s.qb[1] = reinterpret_cast<double*>(take((size_t)3 * n * 8, 16));
    s.dF = reinterpret_cast<double*>(take((size_t)n * 8, 16));
    s.qfb[0] = reinterpret_cast<float4*>(take((size_t)n * 16, 16));
    s.qfb[1] = reinterpret_cast<float4*>(take((size_t)n * 16, 16));
    s.q = s.qb[0];
    s.qf = s.qfb[0];
    s.F = reinterpret_cast<double*>(take((size_t)3 * m * 8, 16));
    s.qref = reinterpret_cast<float4*>(take((size_t)m * 16, 16));
    s.part = reinterpret_cast<double*>(take((size_t)K * 4 * 8, 16));
    s.stale = reinterpret_cast<int*>(take((size_t)K * 4, 16));
    s.nbl = reinterpret_cast<unsigned short*>(take((size_t)m * EAM_LIST_CAP * 2, 16));
    s.nbc = reinterpret_cast<unsigned char*>(take((size_t)2 * m, 16));
    return s;
}

// The cluster's view: rank, owned atoms and the split of the pair entries over S threads.
struct SweepOwn {
    int K, rank, a0, mown, m, S;
};

// Own atoms' Verlet lists (every pair within the reach, in index order; the layout of eam_build_list
// over the m own slots).
__device__ inline void sc_build_lists(const SweepClusterShared& s, const SweepOwn& w, int n, const double box[3],
                                      float reach2, int* status) {
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    for (int li = threadIdx.x; li < w.mown; li += blockDim.x) {
        const int i = w.a0 + li;
        const float4 qi = s.qf[i];
        const int cap = EAM_LIST_CAP / w.S;
        int c[2] = {0, 0};
        for (int j = 0; j < n; ++j) {
            if (j == i || !(r2_f32(mi_f32(qi, s.qf[j], boxf, ibf)) < reach2)) continue;
            const int u = w.S == 2 ? (j & 1) : 0;
            if (c[u] < cap) s.nbl[eam_pidx(li, c[u] * w.S + u, w.m, w.S)] = (unsigned short)j;
            ++c[u];
        }
        if (c[0] > cap || c[1] > cap) flag(status, ST_NEIGH);
        for (int u = 0; u < w.S; ++u) s.nbc[u * w.m + li] = (unsigned char)(c[u] > cap ? cap : c[u]);
        s.qref[li] = qi;
    }
}

// The two EAM pair passes of the own atoms (eam_forces_cta's arithmetic and entry split); the
// F'(rho) of the own atoms go to every CTA before the force pass.  All threads; ends with a CTA
// barrier.
template <typename real>
__device__ void sc_forces(const SweepClusterShared& s, const SweepOwn& w, int n, const double box[3], const FSDev& p,
                          cooperative_groups::cluster_group& cl) {
    EamShared e{};
    e.q = s.q;
    e.qf = s.qf;
    e.dF = s.dF;
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const real d_ = (real)p.d, c_ = (real)p.c, c0 = (real)p.c0, c1 = (real)p.c1, c2 = (real)p.c2;
    const int S = w.S;
    const int span = (S * w.mown + 31) / 32 * 32;
    const int stride = S * w.m;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const int li = t / S, u = t - (t / S) * S;
        const bool act = li < w.mown;
        real rho = 0;
        if (act) {
            const int i = w.a0 + li;
            const float4 qi = s.qf[i];
            const int cnt = s.nbc[u * w.m + li];
            for (int k = 0, o = li * S + u; k < cnt; ++k, o += stride) {
                const int j = s.nbl[o];
                real dv[3], r;
                if (!pair_in<real>(e, n, i, j, qi, box, boxf, ibf, p.screen2, r, dv)) continue;
                if (r < d_) rho += (r - d_) * (r - d_);
            }
        }
        if (S == 2) rho += __shfl_xor_sync(0xffffffffu, rho, 1);
        if (act && u == 0) {
            const int i = w.a0 + li;
            double dF;
            if constexpr (sizeof(real) == 4) dF = rho > 0.f ? (double)(-0.5f * (float)p.A / sqrtf(rho)) : 0.0;
            else dF = (double)rho > 0.0 ? -p.A / (2.0 * sqrt((double)rho)) : 0.0;
            for (int r2 = 0; r2 < w.K; ++r2) cl.map_shared_rank(s.dF, r2)[i] = dF;
        }
    }
    cl.sync();   // every CTA has every F'(rho)
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const int li = t / S, u = t - (t / S) * S;
        const bool act = li < w.mown;
        real f0 = 0, f1 = 0, f2 = 0;
        if (act) {
            const int i = w.a0 + li;
            const real dFi = (real)s.dF[i];
            const float4 qi = s.qf[i];
            const int cnt = s.nbc[u * w.m + li];
            for (int k = 0, o = li * S + u; k < cnt; ++k, o += stride) {
                const int j = s.nbl[o];
                real dv[3], r;
                if (!pair_in<real>(e, n, i, j, qi, box, boxf, ibf, p.screen2, r, dv)) continue;
                eam_pair_force<real>(e, j, r, dv, dFi, d_, c_, c0, c1, c2, f0, f1, f2);
            }
        }
        if (S == 2) {
            f0 += __shfl_xor_sync(0xffffffffu, f0, 1);
            f1 += __shfl_xor_sync(0xffffffffu, f1, 1);
            f2 += __shfl_xor_sync(0xffffffffu, f2, 1);
        }
        if (act && u == 0) {
            s.F[li] = (double)f0;
            s.F[w.m + li] = (double)f1;
            s.F[2 * w.m + li] = (double)f2;
        }
    }
    __syncthreads();
}

// New position of own atom i (rows of q, wrapped copy) into every CTA's other position buffer
// (nb: its index), which becomes the current one after the next cluster barrier.
__device__ __forceinline__ void sc_publish_pos(const SweepClusterShared& s, const SweepOwn& w, int n, int nb, int i,
                                               const double qx, const double qy, const double qz, const float4 qf,
                                               cooperative_groups::cluster_group& cl) {
    for (int r = 0; r < w.K; ++r) {
        double* q = cl.map_shared_rank(s.qb[nb], r);
        q[i] = qx;
        q[n + i] = qy;
        q[2 * n + i] = qz;
        cl.map_shared_rank(s.qfb[nb], r)[i] = qf;
    }
}

// Switch to the buffers published into (after the cluster barrier that follows the publication).
__device__ __forceinline__ void sc_flip(SweepClusterShared& s, int& cb) {
    cb ^= 1;
    s.q = s.qb[cb];
    s.qf = s.qfb[cb];
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

// Every CTA's partial sums (after the cluster barrier) combined in rank order: (a, b, mx, bad).
__device__ __forceinline__ void sc_totals(const SweepClusterShared& s, const SweepOwn& w, double& a, double& b,
                                          double& mx, int& bad) {
    a = 0.0;
    b = 0.0;
    mx = 0.0;
    bad = 0;
    for (int r = 0; r < w.K; ++r) {
        a += s.part[4 * r];
        b += s.part[4 * r + 1];
        mx = fmax(mx, s.part[4 * r + 2]);
        bad |= s.part[4 * r + 3] != 0.0;
    }
}

template <typename real>
__global__ void __launch_bounds__(256, 1) k_parareal_sweep_cluster(
    int n, int m, double b0, double b1, double b2, FSDev fs, LangevinDev L, int nsteps, int n_in, int n_fin,
    const double* __restrict__ jumps, const double* __restrict__ prev, double* __restrict__ cur,
    double* __restrict__ cout, double delta_expl, int metric, const double* __restrict__ Gwin, SweepResult* res,
    int* status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[33];
    SweepOwn w;
    w.K = (int)cl.num_blocks();
    w.rank = (int)cl.block_rank();
    w.m = m;
    w.a0 = w.rank * m;
    w.mown = w.a0 >= n ? 0 : (n - w.a0 < m ? n - w.a0 : m);
    w.S = n <= 256 ? 2 : 1;   // the entry split of the one-CTA kernels' launch shape
    SweepClusterShared s = sweep_cluster_carve(smem, n, m, w.K);
    int cb = 0;   // current position buffer (the same in every CTA: all publish at the same points)
    const double box[3] = {b0, b1, b2};
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const float lim2 = 0.25f * EAM_SKIN * EAM_SKIN;
    const long SS = 6L * n;
    const int t = threadIdx.x;
    const bool mine = t < w.mown;   // thread t integrates own atom a0 + t
    const int i = w.a0 + t;
    // the window's first state: every CTA loads all positions, the own threads their velocities
    for (int x = t; x < 3 * n; x += blockDim.x) s.q[x] = cur[x];
    double v[3] = {0.0, 0.0, 0.0}, vh[3] = {0.0, 0.0, 0.0};
    if (mine)
        for (int al = 0; al < 3; ++al) v[al] = cur[3 * n + al * n + i];
    __syncthreads();
    for (int x = t; x < n; x += blockDim.x) s.qf[x] = wrap_f32(s.q[x], s.q[n + x], s.q[2 * n + x], box);
    __syncthreads();
    // error sums from n = n_in: |q^cur - q^prev| and |q^prev| of the first state
    {
        double a = 0.0, bb = 0.0, mx = 0.0;
        if (mine) {
            double d2 = 0.0;
            for (int al = 0; al < 3; ++al) {
                const double c = cur[al * n + i], pp = prev[al * n + i];
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
    double num = 0.0, den = 0.0, delta;
    {
        double A, B, M;
        int bad;
        sc_totals(s, w, A, B, M, bad);
        if (metric == PMD_METRIC_REL) {
            num = sqrt(A);
            den = sqrt(B);
            delta = den > 0 ? num / den : 0.0;
        } else {
            num = sqrt(M);
            delta = num;
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
        double Jo[6] = {0, 0, 0, 0, 0, 0}, Po[3] = {0, 0, 0};
        if (mine) {
            for (int c = 0; c < 6; ++c) Jo[c] = J ? J[c * n + i] : 0.0;
            for (int al = 0; al < 3; ++al) Po[al] = P[al * n + i];
        }
        // ---- C(cur_n): nsteps sub-steps of interval nn (coarse_interval_cta's arithmetic)
        bool bad = false;
        if (nsteps > 0) {
            double Gc[3] = {0, 0, 0};
            if (mine) coarse_noise<1>(L, Gp, (int64_t)nn, 0, i, n, Gc);
            sc_forces<real>(s, w, n, box, fs, cl);
            if (L.scheme == PMD_SCHEME_PAPER) {
                for (int al = 0; al < 3; ++al) vh[al] = v[al];
                for (int ell = 0; ell < nsteps; ++ell) {
                    const double s0 = sched_sigma(L, ell), s1 = sched_sigma(L, ell + 1);
                    int st = 0;
                    if (mine) {
                        double qn[3];
                        for (int al = 0; al < 3; ++al) {
                            const double vhn = half_kick(L, v[al], s.F[al * m + t], vh[al], s0, Gc[al]);
                            vh[al] = vhn;
                            const double q0 = s.q[al * n + i];
                            qn[al] = drift(q0, L.dt, vhn);
                            if (!isfinite(qn[al])) bad = true;
                            if (fabs(qn[al] - q0) > 0.5 * box[al]) flag(status, ST_LOSTATOM);
                        }
                        const float4 qw = wrap_f32(qn[0], qn[1], qn[2], box);
                        sc_publish_pos(s, w, n, cb ^ 1, i, qn[0], qn[1], qn[2], qw, cl);
                        coarse_noise<1>(L, Gp, (int64_t)nn, ell + 1, i, n, Gc);
                        st = r2_f32(mi_f32(s.qref[t], qw, boxf, ibf)) > lim2;
                    }
                    sc_publish_stale(s, w, st, cl);
                    cl.sync();   // positions and staleness of every atom
                    sc_flip(s, cb);
                    sc_refresh(s, w, n, box, fs, status);
                    sc_forces<real>(s, w, n, box, fs, cl);
                    if (mine)
                        for (int al = 0; al < 3; ++al)
                            v[al] = half_kick(L, vh[al], s.F[al * m + t], vh[al], s1, Gc[al]);
                }
            } else {
                for (int ell = 0; ell < nsteps; ++ell) {
                    int st = 0;
                    if (mine) {
                        double qn[3];
                        for (int al = 0; al < 3; ++al) {
                            double vv = kick_b(L, v[al], s.F[al * m + t]);
                            const double q0 = s.q[al * n + i];
                            double q = __dadd_rn(q0, __dmul_rn(L.hdt, vv));
                            vv = ou_o(L, vv, Gc[al]);
                            q = __dadd_rn(q, __dmul_rn(L.hdt, vv));
                            if (!isfinite(q)) bad = true;
                            if (fabs(q - q0) > 0.5 * box[al]) flag(status, ST_LOSTATOM);
                            qn[al] = q;
                            v[al] = vv;
                        }
                        const float4 qw = wrap_f32(qn[0], qn[1], qn[2], box);
                        sc_publish_pos(s, w, n, cb ^ 1, i, qn[0], qn[1], qn[2], qw, cl);
                        if (ell + 1 < nsteps) coarse_noise<1>(L, Gp, (int64_t)nn, ell + 1, i, n, Gc);
                        st = r2_f32(mi_f32(s.qref[t], qw, boxf, ibf)) > lim2;
                    }
                    sc_publish_stale(s, w, st, cl);
                    cl.sync();
                    sc_flip(s, cb);
                    sc_refresh(s, w, n, box, fs, status);
                    sc_forces<real>(s, w, n, box, fs, cl);
                    if (mine)
                        for (int al = 0; al < 3; ++al) v[al] = kick_b(L, v[al], s.F[al * m + t]);
                }
            }
        }
        if (bad) flag(status, ST_NONFINITE);
        // ---- jump, writes, error sums, and the corrected state to every CTA
        double a = 0.0, bb = 0.0, mx = 0.0;
        int st = 0, nonfin = bad ? 1 : 0;
        if (mine) {
            double d2 = 0.0, qn[3];
            for (int al = 0; al < 3; ++al) {
                const double c = s.q[al * n + i];
                co[al * n + i] = c;
                const double u = J ? c + Jo[al] : c;
                qn[al] = u;
                cn[al * n + i] = u;
                if (!isfinite(u)) nonfin = 1;
                const double pp = Po[al];
                d2 += (u - pp) * (u - pp);
                bb += pp * pp;
            }
            a = d2;
            mx = d2;
            for (int al = 0; al < 3; ++al) {
                const double c = v[al];
                co[3 * n + al * n + i] = c;
                const double u = J ? c + Jo[3 + al] : c;
                v[al] = u;
                cn[3 * n + al * n + i] = u;
                if (!isfinite(u)) nonfin = 1;
            }
            const float4 qw = wrap_f32(qn[0], qn[1], qn[2], box);
            st = r2_f32(mi_f32(s.qref[t], qw, boxf, ibf)) > lim2;
            sc_publish_pos(s, w, n, cb ^ 1, i, qn[0], qn[1], qn[2], qw, cl);
        }
        const double A = cta_sum(a, red), B = cta_sum(bb, red), M = cta_max(mx, red);
        const int anybad = __syncthreads_or(nonfin);
        if (t == 0)
            for (int r = 0; r < w.K; ++r) {
                double* pr = cl.map_shared_rank(s.part, r) + 4 * w.rank;
                pr[0] = A;
                pr[1] = B;
                pr[2] = M;
                pr[3] = anybad ? 1.0 : 0.0;
            }
        sc_publish_stale(s, w, st, cl);
        cl.sync();   // corrected state, partial sums and staleness of every CTA
        sc_flip(s, cb);
        {
            double TA, TB, TM;
            int tbad;
            sc_totals(s, w, TA, TB, TM, tbad);
            if (metric == PMD_METRIC_REL) {
                num += sqrt(TA);
                den += sqrt(TB);
                delta = num / den;
            } else {
                num = fmax(num, sqrt(TM));
                delta = num;
            }
            if (tbad || !isfinite(delta)) delta = INFINITY;
        }
        if (!(delta <= delta_expl)) {
            n_stop = nn;
            break;
        }
        sc_refresh(s, w, n, box, fs, status);
    }
    if (w.rank == 0 && t == 0) {
        res->delta = delta;
        res->n_stop = n_stop;
    }
    cl.sync();   // no CTA leaves while another may still write into its shared memory
}

}  // namespace pmd
