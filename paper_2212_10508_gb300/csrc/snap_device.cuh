// SNAP device helpers (fine potential, Sec. 3.1; method of Thompson et al. 2015): layouts,
// neighbour search, Cayley-Klein parameters and the deterministic force gather.  The per-atom
// pass built on them is in snap_v2.cuh.  The mathematics used there:
//   * U_tot^j = I + sum_k fc(r_k) U^j(a_k, b_k) on the half layout (columns m >= 0), U^j built
//     level by level from U^{j-1/2}:
//       m > 0 : U^j_{m'm} = [a sqrt(j+m') U^{j-1/2}_{m'-1/2,m-1/2} - conj(b) sqrt(j-m') U^{j-1/2}_{m'+1/2,m-1/2}] / sqrt(j+m)
//       m = 0 : U^j_{m'm} = [b sqrt(j+m') U^{j-1/2}_{m'-1/2,m+1/2} + conj(a) sqrt(j-m') U^{j-1/2}_{m'+1/2,m+1/2}] / sqrt(j-m)
//     and mirrored with U_{-m',-m} = (-1)^{m'-m} conj(U_{m'm});
//   * the adjoint Y^J = dE_i/dU^J (dE_i = Re sum conj(Y) dU) as the sum over blocks (a >= b, J)
//     of beta_eff(a,b,J) Z^J_{ab}, Z^J_{ab}(m,m') = sum C^{Jm}_{a m1 b m-m1} C^{Jm'}_{a m1' b m'-m1'}
//     U^a_{m1m1'} U^b_{m-m1,m'-m1'} (the three factors of each B triple folded into one block
//     list through the Clebsch-Gordan symmetries);
//   * per neighbour, dE_i/dr_ik = w Re tr(Y^dag U T_alpha) + (dw/dr_alpha) Re tr(Y^dag U) with
//     T_alpha = drho(g^-1 dg/dr_alpha) tridiagonal in m: only four weighted sums over the half
//     layout (D, P, Q, S0) are needed per neighbour.
// No float atomics: per-pair results are written to fixed slots and gathered in index order.
#pragma once

#include "device_common.cuh"

namespace pmd {

constexpr int NMAX = PMD_MAX_NEIGHBORS;

__host__ __device__ constexpr int h_qlo(int tj) { return (tj + 1) / 2; }
__host__ __device__ constexpr int h_ncol(int tj) { return tj + 1 - (tj + 1) / 2; }
__host__ __device__ constexpr int h_off(int tj) {
    int o = 0;
    for (int t = 0; t < tj; ++t) o += (t + 1) * h_ncol(t);
    return o;
}
__host__ __device__ constexpr int f_off(int tj) { return tj * (tj + 1) * (2 * tj + 1) / 6; }

template <int TJ>
struct Dims {
    static constexpr int NHALF = h_off(TJ + 1);
    static constexpr int NFULL = f_off(TJ + 1);
    static constexpr int NR = (NHALF + 31) / 32;
};

template <typename real>
struct Vec4 {
    real x, y, z, r;
};

struct SnapDevParams {
    float rcut_f;
    double rcut, rfac0;
    int switchflag;
};

// --- positions --------------------------------------------------------------------------
// FP64 path: rows of the member's positions, minimum image with round-to-nearest and no
// contraction (matches the plain FP64 definition exactly).
__device__ __forceinline__ void disp64(const double* q, int n, int i, int k, const double box[3], double d[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = __dsub_rn(q[a * n + k], q[a * n + i]);
        double s = rint(x * (1.0 / box[a]));   // the image of x / box except near half a box length
        d[a] = __dsub_rn(x, __dmul_rn(box[a], s));
    }
}
__device__ __forceinline__ double r2_64(const double d[3]) {
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// --- neighbour search: one warp, one atom --------------------------------------------------
template <typename real>
__device__ __forceinline__ int warp_neighbors(int* nbr, Vec4<real>* disp, int lane, int n, int i,
                                              const double* q64, const float4* qf, const double box[3],
                                              double rcut, int* status) {
    const float boxf0 = (float)box[0], boxf1 = (float)box[1], boxf2 = (float)box[2];
    int cnt = 0;
    const unsigned full = 0xffffffffu;
    if constexpr (sizeof(real) == 8) {
        const double rc2 = rcut * rcut;
        for (int k0 = 0; k0 < n; k0 += 32) {
            int k = k0 + lane;
            bool in = false;
            double d[3] = {0, 0, 0}, r2 = 0;
            if (k < n && k != i) {
                disp64(q64, n, i, k, box, d);
                r2 = r2_64(d);
                in = r2 < rc2;
            }
            unsigned m = __ballot_sync(full, in);
            if (in) {
                int pos = cnt + __popc(m & ((1u << lane) - 1u));
                if (pos < NMAX) {
                    nbr[pos] = k;
                    disp[pos] = Vec4<real>{(real)d[0], (real)d[1], (real)d[2], (real)sqrt(r2)};
                }
            }
            cnt += __popc(m);
        }
    } else {
        const float rc2 = (float)(rcut * rcut);
        const float4 qi = qf[i];
        const float ib0 = 1.0f / boxf0, ib1 = 1.0f / boxf1, ib2 = 1.0f / boxf2;
        for (int k0 = 0; k0 < n; k0 += 32) {
            int k = k0 + lane;
            bool in = false;
            float dx = 0, dy = 0, dz = 0, r2 = 0;
            if (k < n && k != i) {
                float4 qk = qf[k];
                dx = qk.x - qi.x;
                dy = qk.y - qi.y;
                dz = qk.z - qi.z;
                dx -= boxf0 * rintf(dx * ib0);
                dy -= boxf1 * rintf(dy * ib1);
                dz -= boxf2 * rintf(dz * ib2);
                r2 = dx * dx + dy * dy + dz * dz;
                in = r2 < rc2;
            }
            unsigned m = __ballot_sync(full, in);
            if (in) {
                int pos = cnt + __popc(m & ((1u << lane) - 1u));
                if (pos < NMAX) {
                    nbr[pos] = k;
                    disp[pos] = Vec4<real>{(real)dx, (real)dy, (real)dz, (real)sqrtf(r2)};
                }
            }
            cnt += __popc(m);
        }
    }
    if (cnt > NMAX) {
        if (lane == 0) flag(status, ST_NEIGH);
        cnt = NMAX;
    }
    __syncwarp();
    return cnt;
}

// Cayley-Klein parameters of one neighbour: a = cos t - i sin t z/r, b = sin t (y - i x)/r.
template <typename real>
__device__ __forceinline__ void cayley_klein(const Vec4<real>& d, real kappa, real rcut, int sw,
                                             cplx<real>& a, cplx<real>& b, real& w) {
    real s, c;
    if constexpr (sizeof(real) == 8) sincos(kappa * d.r, &s, &c);
    else sincosf(kappa * d.r, &s, &c);
    real ir = real(1) / d.r;
    a = {c, -s * d.z * ir};
    b = {s * d.y * ir, -s * d.x * ir};
    if (sw) {
        if constexpr (sizeof(real) == 8) w = real(0.5) * (cos(real(PI) * d.r / rcut) + real(1));
        else w = 0.5f * (cosf(float(PI) * d.r / rcut) + 1.0f);
    } else {
        w = real(1);
    }
}

// Unevaluated float pair hi + lo (double-float arithmetic, Knuth's TwoSum / Dekker's Fast2Sum):
// used to sum FP32 pair derivatives with FP64-class accuracy on the FP32 pipes.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return FF{s, e};   // s + e == a + b exactly
}
// Symmetric in its arguments (the exact error of hi + hi, then lo + lo, then one renormalisation),
// so a butterfly leaves the same bits in every lane.
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    const float hi = __fadd_rn(s.hi, e);
    return FF{hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}
__device__ __forceinline__ FF ff_shfl_xor(FF x, int m) {
    return FF{__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)};
}

// Slot of atom k in the index-sorted list of j (nbr row lj, cj entries), or -1: from the member's
// slot table pos[j][k] when there is one (written with the lists; checked against the list), else
// by binary search.
__device__ __forceinline__ int reverse_slot(const int* __restrict__ lj, int cj, int j, int k,
                                            const unsigned char* pos, int n) {
    if (pos) {
        const int c = pos[(size_t)j * n + k];
        return (c < cj && lj[c] == k) ? c : -1;
    }
    int lo = 0, hi = cj - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = lj[mid];
        if (v == k) return mid;
        if (v < k) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Force on atom k of a system, one warp: F_k = sum_{j in N(k)} (dE_k/dr_kj - dE_j/dr_jk), with
// neighbour lists sorted by index and symmetric.  Lane l handles the neighbour slots l and l + 32
// of N(k) (the slot of k in N(j): reverse_slot); the per-lane partial sums are combined by a
// butterfly over the 32 lanes: a fixed order, and every lane ends with the same bits.
// FP32 pair derivatives: every difference is held exactly as a float pair and summed in
// double-float arithmetic (F = hi + lo, evaluated in FP64 by the caller); FP64: plain FP64 sums.
__device__ __forceinline__ void warp_gather_force_ff(const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                     const float* __restrict__ dedr, int k, int lane, FF F[3],
                                                     int* status, const unsigned char* pos = nullptr, int n = 0) {
    const int ck = nnb[k];
    const int* lk = nbr + (size_t)k * NMAX;
    const float* dk = dedr + (size_t)k * NMAX * 3;
    FF f[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int s = lane; s < ck; s += 32) {
        const int j = lk[s];
        const int cj = nnb[j];
        const int t = reverse_slot(nbr + (size_t)j * NMAX, cj, j, k, pos, n);
        if (t < 0) flag(status, ST_BADNEIGH);
        const float* dj = dedr + ((size_t)j * NMAX + (t < 0 ? 0 : t)) * 3;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float g = dk[s * 3 + a];
            const float h = t < 0 ? 0.f : dj[a];
            f[a] = ff_add(f[a], ff_two_sum(g, -h));
        }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) f[a] = ff_add(f[a], ff_shfl_xor(f[a], m));
    F[0] = f[0];
    F[1] = f[1];
    F[2] = f[2];
}

template <typename real>
__device__ __forceinline__ void warp_gather_force(const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                  const real* __restrict__ dedr, int k, int lane, double F[3],
                                                  int* status, const unsigned char* pos = nullptr, int n = 0) {
    if constexpr (sizeof(real) == 4) {
        FF f[3];
        warp_gather_force_ff(nbr, nnb, dedr, k, lane, f, status, pos, n);
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] = (double)f[a].hi + (double)f[a].lo;
    } else {
        const int ck = nnb[k];
        const int* lk = nbr + (size_t)k * NMAX;
        const real* dk = dedr + (size_t)k * NMAX * 3;
        double f[3] = {0.0, 0.0, 0.0};
        for (int s = lane; s < ck; s += 32) {
            const int j = lk[s];
            const int cj = nnb[j];
            const int t = reverse_slot(nbr + (size_t)j * NMAX, cj, j, k, pos, n);
            if (t < 0) flag(status, ST_BADNEIGH);
            const real* dj = dedr + ((size_t)j * NMAX + (t < 0 ? 0 : t)) * 3;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double g = (double)dk[s * 3 + a];
                const double h = t < 0 ? 0.0 : (double)dj[a];
                f[a] += g - h;
            }
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) f[a] += __shfl_xor_sync(0xffffffffu, f[a], m);
        F[0] = f[0];
        F[1] = f[1];
        F[2] = f[2];
    }
}

}  // namespace pmd
