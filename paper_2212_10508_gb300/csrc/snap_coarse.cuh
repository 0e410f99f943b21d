// SNAP of a small band limit as the coarse potential of the one-CTA coarse kernels (Strategy I of
// Sec. 3: SNAP-6, 2J = 2, as coarse propagator of a larger SNAP fine potential).  One thread per
// atom, on the CTA-resident state of the coarse path (positions in shared memory, the Verlet
// list of eam_device.cuh built for the SNAP cutoff):
//   pass 1: U_tot^j = I + sum_k fc(r_ik) U^j(a_k, b_k) (the half-layout recursion of snap_v2.cuh,
//           one neighbour after the other, in list order), then Y^J = sum_blocks beta_eff Z^J
//           (every contraction job of the context's table, in table order), kept in shared
//           memory on the half layout;
//   pass 2: F_i = sum_{k in N(i)} (dE_i/dr_ik - dE_k/dr_ki): the thread of atom i evaluates both
//           terms, the second with atom k's Y from shared memory, so every force is a sum in a
//           fixed order with no atomics (each pair term is computed twice, once per end).
// The arithmetic of every term is that of the fine kernels (Cayley-Klein parameters, V = U/nrm
// recursion, the four weighted contractions of the force pass); only the schedule differs.
#pragma once

#include "eam_device.cuh"
#include "snap_v2.cuh"

namespace pmd {

__host__ __device__ constexpr size_t align_up_sz(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device view of a small SNAP context used as coarse potential.
struct SnapCoarseDev {
    const int4* jobs;               // contraction jobs [nrounds][32] (FP64-path layout)
    const unsigned char* round_tb;  // sub-block size of each round
    const void* cg;                 // Clebsch-Gordan values (real)
    const int* beffptr;             // beta_eff = CSR over blocks of (t, coef)
    const int* befft;
    const double* beffc;
    const double* beta;             // [1 + nB] coefficients (engine-owned copy)
    int nrounds, ncg, nblk;
    double rcut, kappa;
    int switchflag;
    float screen2;                  // FP32 screen radius^2 (rcut + margin)
};

// Shared memory of the SNAP coarse passes, after the coarse state: Y of every atom on the half
// layout, beta_eff per block and the Clebsch-Gordan values.
template <typename real, int TJ>
struct SnapCoarseShared {
    cplx<real>* yh;   // [n][NHALF]
    real* beff;       // [nblk]
    real* cg;         // [ncg]
};

template <typename real, int TJ>
__host__ __device__ inline size_t snap_coarse_smem_bytes(int n, int ncg, int nblk) {
    return (size_t)n * Dims<TJ>::NHALF * sizeof(cplx<real>) + align_up_sz((size_t)nblk * sizeof(real), 16) +
           align_up_sz((size_t)ncg * sizeof(real), 16) + 64;
}

template <typename real, int TJ>
__device__ inline SnapCoarseShared<real, TJ> snap_coarse_carve(unsigned char* base, int n, int nblk) {
    SnapCoarseShared<real, TJ> t;
    t.yh = reinterpret_cast<cplx<real>*>(base);
    t.beff = reinterpret_cast<real*>(base + (size_t)n * Dims<TJ>::NHALF * sizeof(cplx<real>));
    t.cg = reinterpret_cast<real*>(reinterpret_cast<unsigned char*>(t.beff) + align_up_sz((size_t)nblk * sizeof(real), 16));
    return t;
}

// beta_eff of every block and the Clebsch-Gordan values into shared memory (all threads; ends
// with a CTA barrier).  Called once per kernel launch.
template <typename real, int TJ>
__device__ inline void snap_coarse_load(const SnapCoarseShared<real, TJ>& t, const SnapCoarseDev& d) {
    for (int b = threadIdx.x; b < d.nblk; b += blockDim.x) {
        double s = 0.0;
        for (int c = d.beffptr[b]; c < d.beffptr[b + 1]; ++c) s += d.beffc[c] * d.beta[1 + d.befft[c]];
        t.beff[b] = (real)s;
    }
    const real* cg = static_cast<const real*>(d.cg);
    for (int x = threadIdx.x; x < d.ncg; x += blockDim.x) t.cg[x] = cg[x];
    __syncthreads();
}

// Sink of the U pass: acc[E] += w V_E (traversal order, half layout).
template <typename real, int TJ>
struct SinkAcc {
    cplx<real>* acc;
    real w;
    template <int E>
    __device__ __forceinline__ void take(cplx<real> v) {
        acc[E].re += w * v.re;
        acc[E].im += w * v.im;
    }
};

// U_tot on the full layout from the weighted V sums: U = nrm V (+1 on the diagonal, the self
// term), mirrored with U_{-m',-m} = (-1)^{m'-m} conj(U_{m'm}).
template <typename real, int TJ>
struct SnapCoarseFin {
    const cplx<real>* acc;
    cplx<real>* U;
    template <int E>
    __device__ __forceinline__ void apply() {
        constexpr HM m = hm(E);
        const real nr = real(m.nrm);
        const cplx<real> v{nr * acc[E].re + (m.p == m.q ? real(1) : real(0)), nr * acc[E].im};
        U[m.full] = v;
        if constexpr (m.mir >= 0) {
            constexpr real sg = m.mirneg ? real(-1) : real(1);
            U[m.mir >= 0 ? m.mir : 0] = {sg * v.re, -sg * v.im};
        }
    }
};

// Pair (i, j) inside the SNAP cutoff: displacement r_j - r_i (exact FP64 minimum image, or the
// FP32 one on wrapped positions) and its length.
template <typename real>
__device__ __forceinline__ bool snap_pair(const EamShared& s, int n, int i, int j, const float4& qi, const double box[3],
                                          const float boxf[3], const float ibf[3], const SnapCoarseDev& d,
                                          Vec4<real>& dv) {
    real r, v[3];
    if (!pair_in<real>(s, n, i, j, qi, box, boxf, ibf, d.screen2, r, v)) return false;
    if constexpr (sizeof(real) == 8) {
        const double dd[3] = {v[0], v[1], v[2]};
        if (!(r2_64(dd) < d.rcut * d.rcut)) return false;
    } else {
        if (!(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] < (float)(d.rcut * d.rcut))) return false;
    }
    dv = Vec4<real>{v[0], v[1], v[2], r};
    return true;
}

// yw[0..3][E] = wD Y, wS Y, wP Y(q+1), wQ Y(q-1) times nrm (traversal order) from Y on the half
// layout (row-major half index): the weighted copies the force pass contracts with V = U / nrm.
template <typename real, int TJ>
struct WeightY {
    const cplx<real>* yh;
    cplx<real>* full;
    cplx<real>* yw;
    template <int E>
    __device__ __forceinline__ void apply() {   // expand to the full layout (mirror images)
        constexpr HM m = hm(E);
        const cplx<real> v = yh[m.hidx];
        full[m.full] = v;
        if constexpr (m.mir >= 0) {
            constexpr real sg = m.mirneg ? real(-1) : real(1);
            full[m.mir >= 0 ? m.mir : 0] = {sg * v.re, -sg * v.im};
        }
    }
};
template <typename real, int TJ>
struct WeightY2 {
    const cplx<real>* full;
    cplx<real>* yw;
    template <int E>
    __device__ __forceinline__ void apply() {
        constexpr HM m = hm(E);
        constexpr int NH = Dims<TJ>::NHALF;
        const cplx<real> y0 = full[m.full];
        const real wD = real(m.wD * m.nrm), wS = real(m.wS * m.nrm), wP = real(m.wP * m.nrm), wQ = real(m.wQ * m.nrm);
        yw[E] = {wD * y0.re, wD * y0.im};
        yw[NH + E] = {wS * y0.re, wS * y0.im};
        const cplx<real> yp = full[m.yp >= 0 ? m.yp : m.full];
        const cplx<real> ym = full[m.ym >= 0 ? m.ym : m.full];
        yw[2 * NH + E] = {wP * yp.re, wP * yp.im};
        yw[3 * NH + E] = {wQ * ym.re, wQ * ym.im};
    }
};

template <typename real, int TJ>
__device__ __forceinline__ void snap_coarse_weights(const cplx<real>* yh, cplx<real>* yw) {
    cplx<real> full[Dims<TJ>::NFULL];
    WeightY<real, TJ> a{yh, full, yw};
    ForE<0, Dims<TJ>::NHALF>::run(a);
    WeightY2<real, TJ> b{full, yw};
    ForE<0, Dims<TJ>::NHALF>::run(b);
}

// dE_i/dr_ik of one pair (displacement d = r_k - r_i) against the weighted copies yw of Y_i.
template <typename real, int TJ>
__device__ __forceinline__ void snap_coarse_dedr(const Vec4<real>& d, const cplx<real>* yw, const SnapCoarseDev& c,
                                                 real out[3]) {
    const real kappa = (real)c.kappa, rcut = (real)c.rcut;
    cplx<real> a, b;
    real w;
    cayley_klein<real>(d, kappa, rcut, c.switchflag, a, b, w);
    SinkF<real, TJ> sink{yw};
    URec<real, TJ, SinkF<real, TJ>> rec(a, b, sink);
    ForE<0, Dims<TJ>::NHALF>::run(rec);
    dedr_lane<real>(d, kappa, rcut, c.switchflag, a, b, w, sink.Dim, sink.Sre, sink.Pre, sink.Pim, sink.Qre, sink.Qim,
                    out);
}

// Forces of the SNAP coarse potential into s.F.  All threads of the CTA call it; the caller keeps
// the Verlet list valid for the SNAP cutoff.  Ends with a CTA barrier.
template <typename real, int TJ>
__device__ void snap_coarse_forces_cta(const EamShared& s, const SnapCoarseShared<real, TJ>& t, int n,
                                       const double box[3], const SnapCoarseDev& c) {
    constexpr int NH = Dims<TJ>::NHALF, NF = Dims<TJ>::NFULL;
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const int S = eam_split(n);
    const real kappa = (real)c.kappa, rcut = (real)c.rcut;
    // pass 1: U_tot and Y of atom i
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 qi = s.qf[i];
        cplx<real> acc[NH];
#pragma unroll
        for (int e = 0; e < NH; ++e) acc[e] = {real(0), real(0)};
        for (int u = 0, k = 0; u < S; k = 0, ++u)   // the S sub-lists in turn (see eam_build_list)
        for (; k < s.nbc[u * n + i]; ++k) {
            const int j = s.nbl[eam_pidx(i, k * S + u, n, S)];
            Vec4<real> dv;
            if (!snap_pair<real>(s, n, i, j, qi, box, boxf, ibf, c, dv)) continue;
            cplx<real> a, b;
            real w;
            cayley_klein<real>(dv, kappa, rcut, c.switchflag, a, b, w);
            SinkAcc<real, TJ> sink{acc, w};
            URec<real, TJ, SinkAcc<real, TJ>> rec(a, b, sink);
            ForE<0, NH>::run(rec);
        }
        cplx<real> U[NF];
        SnapCoarseFin<real, TJ> fin{acc, U};   // V -> U, the self term on the diagonal, mirror images
        ForE<0, NH>::run(fin);
        cplx<real> yh[NH + 1];
#pragma unroll
        for (int e = 0; e <= NH; ++e) yh[e] = {real(0), real(0)};
        for (int r = 0; r < c.nrounds; ++r) {
            const int tb = c.round_tb[r];
            for (int l = 0; l < 32; ++l) {
                const int4 J = c.jobs[r * 32 + l];
                if (tb == 0) y_job<real, 0>(J, U, t.cg, t.beff, yh);
                else if (tb == 1) y_job<real, 1>(J, U, t.cg, t.beff, yh);
                else if constexpr (TJ >= 2) y_job<real, (TJ >= 2 ? 2 : 1)>(J, U, t.cg, t.beff, yh);
            }
        }
#pragma unroll
        for (int e = 0; e < NH; ++e) t.yh[(size_t)i * NH + e] = yh[e];
    }
    __syncthreads();
    // pass 2: F_i = sum_k (dE_i/dr_ik - dE_k/dr_ki)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 qi = s.qf[i];
        cplx<real> ywi[4 * NH];
        snap_coarse_weights<real, TJ>(t.yh + (size_t)i * NH, ywi);
        double f[3] = {0.0, 0.0, 0.0};
        for (int u = 0, kk = 0; u < S; kk = 0, ++u)   // the S sub-lists in turn
        for (; kk < s.nbc[u * n + i]; ++kk) {
            const int k = s.nbl[eam_pidx(i, kk * S + u, n, S)];
            Vec4<real> dv;
            if (!snap_pair<real>(s, n, i, k, qi, box, boxf, ibf, c, dv)) continue;
            real g[3], h[3];
            snap_coarse_dedr<real, TJ>(dv, ywi, c, g);
            cplx<real> ywk[4 * NH];
            snap_coarse_weights<real, TJ>(t.yh + (size_t)k * NH, ywk);
            const Vec4<real> dr{-dv.x, -dv.y, -dv.z, dv.r};
            snap_coarse_dedr<real, TJ>(dr, ywk, c, h);
#pragma unroll
            for (int a = 0; a < 3; ++a) f[a] += (double)g[a] - (double)h[a];
        }
        s.F[i] = f[0];
        s.F[n + i] = f[1];
        s.F[2 * n + i] = f[2];
    }
    __syncthreads();
}

// Keep the Verlet list valid for the SNAP cutoff (rebuild when stale or not built yet).
__device__ __forceinline__ void snap_coarse_refresh_list(const EamShared& s, int n, const double box[3],
                                                         const SnapCoarseDev& c, bool force_build, int* status) {
    const int stale = force_build ? 1 : eam_list_stale(s, n, box);
    if (stale) {
        __shared__ int overflow;
        if (threadIdx.x == 0) overflow = 0;
        __syncthreads();
        const float reach = sqrtf(c.screen2) + EAM_SKIN;
        eam_build_list(s, n, box, reach * reach, &overflow);
        __syncthreads();
        if (overflow && threadIdx.x == 0) flag(status, ST_NEIGH);
        __syncthreads();
    }
}

}  // namespace pmd
