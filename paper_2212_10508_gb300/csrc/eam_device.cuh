// Finnis-Sinclair EAM on one system per CTA (coarse potential, Sec. 3.1):
//   rho_i = sum_{j != i, r < d} (r - d)^2,
//   E = sum_i -A sqrt(rho_i) + 1/2 sum_{i != j, r < c} (r - c)^2 (c0 + c1 r + c2 r^2),
//   F_i = sum_j [ (F'(rho_i) + F'(rho_j)) 2 (r - d) [r<d] + phi'(r) [r<c] ] (r_j - r_i) / r,
//   F'(rho) = -A / (2 sqrt rho), 0 when rho = 0.
// Positions live in shared memory (FP64 rows plus a wrapped FP32 copy used to screen pairs).
// FP64 mode evaluates every pair term in FP64 from the exact minimum-image displacement;
// FP32_BULK evaluates pair terms, per-atom sums and the embedding derivative in FP32.
#pragma once

#include "device_common.cuh"
#include "snap_device.cuh"   // disp64 / r2_64

namespace pmd {

struct FSDev {
    double d, A, c, c0, c1, c2;
    float screen2;   // (max(d, c) + margin)^2 for the FP32 screen
};

struct EamShared {
    double* q;                 // [3][n]
    float4* qf;                // [n] wrapped to [0, L)
    double* F;                 // [3][n]
    double* dF;                // [n]
    unsigned short* nbl;       // Verlet list, EAM_LIST_CAP slots per atom (EAM_LIST_CAP / S per sub-list),
                               // eam_pidx layout (nullptr: scan all atoms)
    unsigned char* nbc;        // [S][n] lengths of the per-thread sub-lists (see eam_build_list)
    float4* qref;              // [n] wrapped positions at the last list build
    float4* pg;                // FP32 pair geometry (dx, dy, dz, r) of the density pass, EAM_PG_CAP per atom,
                               // eam_pidx layout
    unsigned short* pj;        // its neighbour indices (nullptr: no cache)
    unsigned char* pgc;        // [n][2] entries per thread slot, EAM_PG_FULL when a slot overflowed
};

// Verlet list of the one-CTA coarse path: every pair within max(d, c) + EAM_SKIN, rebuilt when an
// atom has moved more than EAM_SKIN / 2 since the last build.  With S threads per atom the list
// is S sub-lists, one per thread: thread u of atom i gets the neighbours j with j mod S = u, in
// index order (entry k of sub-list u in slot eam_pidx(i, k S + u, n, S)).  The pair passes
// re-apply the exact cutoff test, so every thread sums the same terms in the same order whatever
// the list's history (a list kept from earlier positions holds extra, rejected entries) and as a
// scan over all atoms: C(x) is the same bits in the sweep, which keeps its list across intervals,
// and in the batch, which builds a fresh one.
constexpr int EAM_LIST_CAP = 64;   // a sub-list longer than EAM_LIST_CAP / S sets ST_NEIGH (ENEIGH)
constexpr float EAM_SKIN = 0.5f;

// FP32 pairs within the screen radius kept from the density pass for the force pass: up to
// EAM_PG_CAP per atom (EAM_PG_CAP / S per thread, k-th pair of thread u of atom i in slot
// eam_pidx(i, u + k S, n, S)); a thread whose pairs do not fit recomputes them in the force pass,
// with the same arithmetic.
constexpr int EAM_PG_CAP = 24;
constexpr unsigned char EAM_PG_FULL = 255;

// Threads per atom in the pair passes of a CTA of blockDim.x threads: two when there are at least
// 2n threads (thread u of atom i takes the neighbours j with j mod 2 = u), one otherwise.
__device__ __forceinline__ int eam_split(int n) { return (int)blockDim.x >= 2 * n ? 2 : 1; }

// Slot of pair entry c of atom i in the list and the pair cache: [c / S][i][c % S], so that the
// threads of consecutive atoms, which walk their entries in step, read consecutive elements
// (no shared-memory bank conflicts).
__device__ __forceinline__ int eam_pidx(int i, int c, int n, int S) {
    const int k = S == 2 ? c >> 1 : c;
    return k * (S * n) + i * S + (c - k * S);
}

// Position wrapped to [0, L) per axis (up to rounding) as FP32: x - L floor(x / L), with the
// quotient taken as x * (1/L), iL = 1/L (the reciprocals are loop invariants of every caller).
// wrap1_f32 is one coordinate; wrap_f32 the three, with the same operations.
__device__ __forceinline__ float wrap1_f32(double x, double L, double iL) {
    x -= L * floor(x * iL);
    return (float)x;
}
__device__ __forceinline__ float4 wrap_f32(double x, double y, double z, const double box[3]) {
    return make_float4(wrap1_f32(x, box[0], 1.0 / box[0]), wrap1_f32(y, box[1], 1.0 / box[1]),
                       wrap1_f32(z, box[2], 1.0 / box[2]), 0.f);
}

// FP32 minimum-image displacement b - a (ibf: reciprocal box lengths; the image only differs
// from the one of a division for pairs near half a box length, far outside every cutoff).
__device__ __forceinline__ float3 mi_f32(const float4& a, const float4& b, const float boxf[3], const float ibf[3]) {
    float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    dx -= boxf[0] * rintf(dx * ibf[0]);
    dy -= boxf[1] * rintf(dy * ibf[1]);
    dz -= boxf[2] * rintf(dz * ibf[2]);
    return make_float3(dx, dy, dz);
}
__device__ __forceinline__ float r2_f32(const float3& d) { return d.x * d.x + d.y * d.y + d.z * d.z; }

// Pair (i, j) if within the screen radius: r and the displacement r_j - r_i in the chosen precision
// (FP32: the screened FP32 displacement itself; FP64: the exact minimum image).  False otherwise.
template <typename real>
__device__ __forceinline__ bool pair_in(const EamShared& s, int n, int i, int j, const float4& qi, const double box[3],
                                        const float boxf[3], const float ibf[3], float screen2, real& r, real d[3]) {
    if (j == i) return false;
    const float3 df = mi_f32(qi, s.qf[j], boxf, ibf);
    const float r2 = r2_f32(df);
    if (!(r2 < screen2)) return false;
    if constexpr (sizeof(real) == 8) {
        double dd[3];
        disp64(s.q, n, i, j, box, dd);
        d[0] = dd[0];
        d[1] = dd[1];
        d[2] = dd[2];
        r = sqrt(r2_64(dd));
    } else {
        d[0] = df.x;
        d[1] = df.y;
        d[2] = df.z;
        r = sqrtf(r2);
    }
    return true;
}

__device__ __forceinline__ void eam_build_list(const EamShared& s, int n, const double box[3], float reach2,
                                               int* overflow) {
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const int S = eam_split(n), cap = EAM_LIST_CAP / S;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 qi = s.qf[i];
        int c[2] = {0, 0};
        for (int j = 0; j < n; ++j) {
            if (j == i || !(r2_f32(mi_f32(qi, s.qf[j], boxf, ibf)) < reach2)) continue;
            const int u = S == 2 ? (j & 1) : 0;
            if (c[u] < cap) s.nbl[eam_pidx(i, c[u] * S + u, n, S)] = (unsigned short)j;
            ++c[u];
        }
        if (c[0] > cap || c[1] > cap) atomicOr(overflow, 1);
        for (int u = 0; u < S; ++u) s.nbc[u * n + i] = (unsigned char)(c[u] > cap ? cap : c[u]);
        s.qref[i] = qi;
    }
}

// 1 when some atom moved more than half the skin since the list was built (CTA-uniform); the
// displacement is taken with the minimum image, so that crossing a face of the box (a jump of
// the wrapped position by a box length) is not a move
__device__ __forceinline__ int eam_list_stale(const EamShared& s, int n, const double box[3]) {
    int stale = 0;
    const float lim2 = 0.25f * EAM_SKIN * EAM_SKIN;
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (r2_f32(mi_f32(s.qref[i], s.qf[i], boxf, ibf)) > lim2) stale = 1;
    return __syncthreads_or(stale);
}

// Pair (i, j) at distance r: g = (dE/dr) / r, the factor of the force g (r_j - r_i) on atom i, from
// the pair term and the embedding derivatives F'(rho_i) = dFi and F'(rho_j); false when r is beyond
// both the density and the pair range (no force).
template <typename real>
__device__ __forceinline__ bool eam_pair_g(real r, real dFi, real dFj, real d_, real c_, real c0, real c1, real c2,
                                           real& g) {
    real dEdr = real(0);
    if (r < d_) dEdr += (dFi + dFj) * real(2) * (r - d_);
    if (r < c_) dEdr += real(2) * (r - c_) * (c0 + c1 * r + c2 * r * r) + (r - c_) * (r - c_) * (c1 + real(2) * c2 * r);
    if (r < d_ || r < c_) {
        g = dEdr / r;
        return true;
    }
    return false;
}

// Adds the pair's force on atom i, g (r_j - r_i), to (f0, f1, f2) (nothing outside both ranges).
template <typename real>
__device__ __forceinline__ void eam_pair_force(const EamShared& s, int j, real r, const real dv[3], real dFi, real d_,
                                               real c_, real c0, real c1, real c2, real& f0, real& f1, real& f2) {
    real g;
    if (eam_pair_g<real>(r, dFi, (real)s.dF[j], d_, c_, c0, c1, c2, g)) {
        f0 += g * dv[0];
        f1 += g * dv[1];
        f2 += g * dv[2];
    }
}

// Forces into s.F (and per-atom energies into Eat if non-null).  All threads of the CTA call it
// (blockDim a multiple of 32); it ends with __syncthreads().  With a list (s.nbl != nullptr) the
// caller keeps it valid (eam_refresh_list); otherwise every atom is scanned.  FP64 accumulates in
// double, FP32_BULK in float (pair terms and sums).  PGCACHE compiles in the pair-geometry cache
// (used when the shared layout has one, FP32 only): the force pass then reads the pairs of the
// density pass instead of screening the list again, with the same bits.
template <typename real, bool PGCACHE = false>
__device__ __forceinline__ void eam_forces_cta(const EamShared& s, int n, const double box[3], const FSDev& p, double* Eat) {
    const float boxf[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float ibf[3] = {1.0f / boxf[0], 1.0f / boxf[1], 1.0f / boxf[2]};
    const real d_ = (real)p.d, c_ = (real)p.c, c0 = (real)p.c0, c1 = (real)p.c1, c2 = (real)p.c2;
    const bool list = s.nbl != nullptr;
    const bool cache = PGCACHE && sizeof(real) == 4 && s.pj != nullptr;
    // S threads per atom when the CTA has at least 2n threads (the launch shape decides; every
    // coarse kernel uses the same one): thread u of atom i sums over the neighbours j = u mod S,
    // and the two partial sums are combined by an xor-shuffle (symmetric: both threads hold the
    // same bits).  span covers whole warps so that every lane takes part in the shuffles.
    const int S = eam_split(n);
    const int span = (S * n + 31) / 32 * 32;
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const int i = t / S, u = t - (t / S) * S;
        const bool act = i < n;
        real rho = 0, ep = 0;
        if (act) {
            const float4 qi = s.qf[i];
            // this thread's neighbours j = u mod S: its sub-list, or every S-th atom without a list
            const int cnt = list ? s.nbc[u * n + i] : (n - u + S - 1) / S;
            const int cap = EAM_PG_CAP / S, stride = S * n;
            int np = 0;
            for (int k = 0, o = i * S + u; k < cnt; ++k, o += stride) {   // o = eam_pidx(i, k S + u, n, S)
                const int j = list ? s.nbl[o] : k * S + u;
                real dv[3], r;
                if (!pair_in<real>(s, n, i, j, qi, box, boxf, ibf, p.screen2, r, dv)) continue;
                if constexpr (sizeof(real) == 4) {
                    if (cache && np < cap) {
                        s.pg[np * stride + i * S + u] = make_float4(dv[0], dv[1], dv[2], r);
                        s.pj[np * stride + i * S + u] = (unsigned short)j;
                    }
                    ++np;
                }
                if (r < d_) rho += (r - d_) * (r - d_);
                if (r < c_) ep += real(0.5) * ((r - c_) * (r - c_) * (c0 + c1 * r + c2 * r * r));
            }
            if (cache) s.pgc[2 * i + u] = np > cap ? EAM_PG_FULL : (unsigned char)np;
        }
        if (S == 2) {
            rho += __shfl_xor_sync(0xffffffffu, rho, 1);
            ep += __shfl_xor_sync(0xffffffffu, ep, 1);
        }
        if (act && u == 0) {
            const double rh = (double)rho;
            if constexpr (sizeof(real) == 4)   // FP32_BULK: the embedding derivative in FP32 as well
                s.dF[i] = rho > 0.f ? (double)(-0.5f * (float)p.A / sqrtf(rho)) : 0.0;
            else
                s.dF[i] = rh > 0.0 ? -p.A / (2.0 * sqrt(rh)) : 0.0;
            if (Eat) Eat[i] = (double)ep - p.A * sqrt(rh);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
        const int i = t / S, u = t - (t / S) * S;
        const bool act = i < n;
        real f0 = 0, f1 = 0, f2 = 0;
        if (act) {
            const real dFi = (real)s.dF[i];
            const int np = cache ? s.pgc[2 * i + u] : EAM_PG_FULL;
            const int stride = S * n;
            if (np != EAM_PG_FULL) {   // the pairs of the density pass, in the same order
#pragma unroll 1
                for (int k = 0, o = i * S + u; k < np; ++k, o += stride) {
                    const float4 g = s.pg[o];
                    const real dv[3] = {(real)g.x, (real)g.y, (real)g.z};
                    eam_pair_force<real>(s, s.pj[o], (real)g.w, dv, dFi, d_, c_, c0, c1, c2, f0, f1, f2);
                }
            } else {
                const float4 qi = s.qf[i];
                const int cnt = list ? s.nbc[u * n + i] : (n - u + S - 1) / S;
                for (int k = 0, o = i * S + u; k < cnt; ++k, o += stride) {
                    const int j = list ? s.nbl[o] : k * S + u;
                    real dv[3], r;
                    if (!pair_in<real>(s, n, i, j, qi, box, boxf, ibf, p.screen2, r, dv)) continue;
                    eam_pair_force<real>(s, j, r, dv, dFi, d_, c_, c0, c1, c2, f0, f1, f2);
                }
            }
        }
        if (S == 2) {
            f0 += __shfl_xor_sync(0xffffffffu, f0, 1);
            f1 += __shfl_xor_sync(0xffffffffu, f1, 1);
            f2 += __shfl_xor_sync(0xffffffffu, f2, 1);
        }
        if (act && u == 0) {
            s.F[i] = (double)f0;
            s.F[n + i] = (double)f1;
            s.F[2 * n + i] = (double)f2;
        }
    }
    __syncthreads();
}

// Keep the Verlet list valid for the current positions (rebuild when stale or not built yet).
__device__ __forceinline__ void eam_refresh_list(const EamShared& s, int n, const double box[3], const FSDev& p,
                                                 bool force_build, int* status) {
    if (!s.nbl) return;
    const int stale = force_build ? 1 : eam_list_stale(s, n, box);
    if (stale) {
        __shared__ int overflow;
        if (threadIdx.x == 0) overflow = 0;
        __syncthreads();
        const float reach = sqrtf(p.screen2) + EAM_SKIN;
        eam_build_list(s, n, box, reach * reach, &overflow);
        __syncthreads();
        if (overflow && threadIdx.x == 0) flag(status, ST_NEIGH);
        __syncthreads();
    }
}

}  // namespace pmd
