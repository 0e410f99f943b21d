// SNAP device code (fine potential, Sec. 3.1; method of Thompson et al. 2015).
//
// One warp handles one atom i:
//   1. neighbour search over the atom's system (ballot-compacted, sorted by index);
//   2. U_tot^j = I + sum_k fc(r_k) U^j(a_k, b_k), accumulated in registers on the half
//      layout (columns m >= 0), U^j built level by level from U^{j-1/2}:
//        m > 0 : U^j_{m'm} = [a sqrt(j+m') U^{j-1/2}_{m'-1/2,m-1/2} - conj(b) sqrt(j-m') U^{j-1/2}_{m'+1/2,m-1/2}] / sqrt(j+m)
//        m = 0 : U^j_{m'm} = [b sqrt(j+m') U^{j-1/2}_{m'-1/2,m+1/2} + conj(a) sqrt(j-m') U^{j-1/2}_{m'+1/2,m+1/2}] / sqrt(j-m)
//      and mirrored with U_{-m',-m} = (-1)^{m'-m} conj(U_{m'm});
//   3. the adjoint Y^J = dE_i/dU^J (dE_i = Re sum conj(Y) dU) as sum over blocks (a >= b, J)
//      of beta_eff(a,b,J) Z^J_{ab}, Z^J_{ab}(m,m') = sum C^{Jm}_{a m1 b m-m1} C^{Jm'}_{a m1' b m'-m1'}
//      U^a_{m1m1'} U^b_{m-m1,m'-m1'} (the three factors of each B triple folded into one
//      block list through the Clebsch-Gordan symmetries);
//   4. per neighbour, dE_i/dr_ik = w Re tr(Y^dag U T_alpha) + (dw/dr_alpha) Re tr(Y^dag U) with
//      T_alpha = drho(g^-1 dg/dr_alpha) tridiagonal in m: only four weighted sums over the
//      half layout (D, P, Q, S0) are needed per neighbour.
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

// per half-layout element (tj, p, q): recursion sources/coefficients and force-pass weights
template <typename real>
struct UElem {
    int src1, src2;      // half indices in level tj-1
    int ufull, umir;     // full index of (p,q) and of its mirror (tj-p, tj-q) (-1: none)
    int y0, yp, ym;      // full indices of (p,q), (p,q+1), (p,q-1) (dummy = y0 when absent)
    int flags;           // bit0: m = 0 rule (b, conj a); bit1: mirror sign is -1
    real c1, c2;         // recursion coefficients
    real cD, cP, cQ, cS; // w(q) m, w(q) sqrt((q+1)(tj-q)), w(q) sqrt((tj-q+1) q), w(q)
};

template <typename real>
struct Vec4 {
    real x, y, z, r;
};

template <typename real, int TJ>
struct WarpScratch {
    int nbr[NMAX];
    Vec4<real> disp[NMAX];
    cplx<real> ulev[Dims<TJ>::NHALF];
    cplx<real> yh[Dims<TJ>::NHALF];
    cplx<real> full[Dims<TJ>::NFULL];   // U_tot, later overwritten by Y
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
        double s = rint(x / box[a]);
        d[a] = __dsub_rn(x, __dmul_rn(box[a], s));
    }
}
__device__ __forceinline__ double r2_64(const double d[3]) {
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// --- neighbour search: one warp, one atom --------------------------------------------------
template <typename real, int TJ>
__device__ __forceinline__ int warp_neighbors(WarpScratch<real, TJ>& ws, int lane, int n, int i,
                                              const double* q64, const float4* qf, const double box[3],
                                              float boxf0, float boxf1, float boxf2, double rcut,
                                              int* status) {
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
                    ws.nbr[pos] = k;
                    ws.disp[pos] = Vec4<real>{(real)d[0], (real)d[1], (real)d[2], (real)sqrt(r2)};
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
                    ws.nbr[pos] = k;
                    ws.disp[pos] = Vec4<real>{(real)dx, (real)dy, (real)dz, (real)sqrtf(r2)};
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

// Build level tj of U(a, b) for the lane's elements into ulev and hand each value to f(r, e, val).
template <typename real, int TJ, typename F>
__device__ __forceinline__ void u_levels(const UElem<real>* __restrict__ elem, cplx<real>* ulev, int lane,
                                         cplx<real> a, cplx<real> b, F&& f) {
    constexpr int NR = Dims<TJ>::NR;
    if (lane == 0) {
        cplx<real> one{real(1), real(0)};
        ulev[0] = one;
        f(0, 0, one);
    }
    __syncwarp();
    const cplx<real> cb{b.re, -b.im};
    const cplx<real> ca{a.re, -a.im};
#pragma unroll
    for (int tj = 1; tj <= TJ; ++tj) {
        const int lo = h_off(tj), hi = h_off(tj + 1);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (32 * r + 31 >= lo && 32 * r < hi) {
                const int e = lane + 32 * r;
                if (e >= lo && e < hi) {
                    const UElem<real>& el = elem[e];
                    cplx<real> u1 = ulev[el.src1], u2 = ulev[el.src2];
                    cplx<real> A1, A2;
                    if (el.flags & 1) {   // m = 0: (b, conj a)
                        A1 = b;
                        A2 = ca;
                    } else {              // m > 0: (a, -conj b)
                        A1 = a;
                        A2 = {-cb.re, -cb.im};
                    }
                    cplx<real> t1 = cmul(A1, u1), t2 = cmul(A2, u2);
                    cplx<real> v{el.c1 * t1.re + el.c2 * t2.re, el.c1 * t1.im + el.c2 * t2.im};
                    ulev[e] = v;
                    f(r, e, v);
                }
            }
        }
        __syncwarp();
    }
}

template <typename real>
__device__ __forceinline__ real warp_sum(real v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// --- the per-atom pass ---------------------------------------------------------------------
// Writes nbr_out[0..cnt), *nnb_out = cnt, dedr_out[slot][3] = dE_i/d r_ik (r_ik = r_k - r_i);
// optionally utot_out[NFULL] (U_tot, full layout) for the energy path.
template <typename real, int TJ>
__device__ void snap_atom_warp(WarpScratch<real, TJ>& ws, const UElem<real>* __restrict__ elem,
                               const int4* __restrict__ jobs, const int* __restrict__ lane_begin,
                               const real* __restrict__ cg, const real* __restrict__ beff,
                               const SnapDevParams& sp, int lane, int n, int i, const double* q64,
                               const float4* qf, const double box[3], int* nbr_out, int* nnb_out,
                               real* dedr_out, cplx<real>* utot_out, int* status) {
    constexpr int NR = Dims<TJ>::NR;
    const real kappa = real(sp.rfac0 * PI / sp.rcut);
    const real rcut = real(sp.rcut);
    const int cnt = warp_neighbors<real, TJ>(ws, lane, n, i, q64, qf, box, (float)box[0], (float)box[1],
                                             (float)box[2], sp.rcut, status);
    for (int s = lane; s < cnt; s += 32) nbr_out[s] = ws.nbr[s];
    if (lane == 0) *nnb_out = cnt;

    // ---- U_tot (half layout, lane-owned registers), self term = identity
    cplx<real> acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int e = lane + 32 * r;
        acc[r] = {real(0), real(0)};
        if (e < Dims<TJ>::NHALF) {
            const UElem<real>& el = elem[e];
            // diagonal element of its level: p == q  <=>  the full index sits on the diagonal
            int tj = 0;
            while (tj < TJ && e >= h_off(tj + 1)) ++tj;
            const int loc = e - h_off(tj);
            const int p = loc / h_ncol(tj), q = h_qlo(tj) + loc % h_ncol(tj);
            if (p == q) acc[r].re = real(1);
            (void)el;
        }
    }
    for (int s = 0; s < cnt; ++s) {
        cplx<real> a, b;
        real w;
        cayley_klein<real>(ws.disp[s], kappa, rcut, sp.switchflag, a, b, w);
        u_levels<real, TJ>(elem, ws.ulev, lane, a, b, [&](int r, int e, cplx<real> v) {
            acc[r].re += w * v.re;
            acc[r].im += w * v.im;
        });
    }
    // write U_tot in full layout (mirror for m > 0)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int e = lane + 32 * r;
        if (e < Dims<TJ>::NHALF) {
            const UElem<real>& el = elem[e];
            ws.full[el.ufull] = acc[r];
            if (el.umir >= 0) {
                real sg = (el.flags & 2) ? real(-1) : real(1);
                ws.full[el.umir] = {sg * acc[r].re, -sg * acc[r].im};
            }
        }
    }
    __syncwarp();
    if (utot_out) {
        for (int e = lane; e < Dims<TJ>::NFULL; e += 32) utot_out[e] = ws.full[e];
    }

    // ---- Y = sum over blocks of beta_eff * Z (lane-owned Y half elements)
    {
        const int jb = lane_begin[lane], je = lane_begin[lane + 1];
        int cur = -1;
        cplx<real> y{real(0), real(0)};
        for (int jj = jb; jj < je; ++jj) {
            const int4 J = jobs[jj];
            const int e = J.x & 0xffff, blk = J.x >> 16;
            const int p = (J.y >> 5) & 31, q = (J.y >> 10) & 31, s = (J.y >> 15) & 31;
            const int ta = (J.y >> 20) & 31, tb = (J.y >> 25) & 31;
            const int ua = J.z & 0xffff, ub = J.z >> 16;
            const real* c = cg + J.w;
            if (e != cur) {
                if (cur >= 0) ws.yh[cur] = y;
                cur = e;
                y = {real(0), real(0)};
            }
            const int p1lo = max(0, p + s - tb), p1hi = min(ta, p + s);
            const int q1lo = max(0, q + s - tb), q1hi = min(ta, q + s);
            cplx<real> z{real(0), real(0)};
            for (int p1 = p1lo; p1 <= p1hi; ++p1) {
                const int p2 = p + s - p1;
                const real c1 = c[p1 * (tb + 1) + p2];
                const cplx<real>* Ua = ws.full + ua + p1 * (ta + 1);
                const cplx<real>* Ub = ws.full + ub + p2 * (tb + 1);
                cplx<real> t{real(0), real(0)};
                for (int q1 = q1lo; q1 <= q1hi; ++q1) {
                    const int q2 = q + s - q1;
                    const real c2 = c[q1 * (tb + 1) + q2];
                    cplx<real> uu = cmul(Ua[q1], Ub[q2]);
                    t.re += c2 * uu.re;
                    t.im += c2 * uu.im;
                }
                z.re += c1 * t.re;
                z.im += c1 * t.im;
            }
            const real be = beff[blk];
            y.re += be * z.re;
            y.im += be * z.im;
        }
        if (cur >= 0) ws.yh[cur] = y;
    }
    __syncwarp();
    // expand Y into the full layout (overwrites U_tot, no longer needed)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int e = lane + 32 * r;
        if (e < Dims<TJ>::NHALF) {
            const UElem<real>& el = elem[e];
            cplx<real> v = ws.yh[e];
            ws.full[el.ufull] = v;
            if (el.umir >= 0) {
                real sg = (el.flags & 2) ? real(-1) : real(1);
                ws.full[el.umir] = {sg * v.re, -sg * v.im};
            }
        }
    }
    __syncwarp();

    // ---- dE_i / d r_ik for every neighbour
    for (int s = 0; s < cnt; ++s) {
        const Vec4<real> d = ws.disp[s];
        cplx<real> a, b;
        real w;
        cayley_klein<real>(d, kappa, rcut, sp.switchflag, a, b, w);
        real Dre = 0, Dim = 0, Pre = 0, Pim = 0, Qre = 0, Qim = 0, Sre = 0;
        u_levels<real, TJ>(elem, ws.ulev, lane, a, b, [&](int, int e, cplx<real> u) {
            const UElem<real>& el = elem[e];
            cplx<real> t0 = cmulc(ws.full[el.y0], u);
            cplx<real> tp = cmulc(ws.full[el.yp], u);
            cplx<real> tm = cmulc(ws.full[el.ym], u);
            Dre += el.cD * t0.re;
            Dim += el.cD * t0.im;
            Sre += el.cS * t0.re;
            Pre += el.cP * tp.re;
            Pim += el.cP * tp.im;
            Qre += el.cQ * tm.re;
            Qim += el.cQ * tm.im;
        });
        Dim = warp_sum(Dim);
        Pre = warp_sum(Pre);
        Pim = warp_sum(Pim);
        Qre = warp_sum(Qre);
        Qim = warp_sum(Qim);
        Sre = warp_sum(Sre);
        (void)Dre;
        if (lane < 3) {
            const int al = lane;
            const real ir = real(1) / d.r;
            const real nx = d.x * ir, ny = d.y * ir, nz = d.z * ir;
            const real na = al == 0 ? nx : (al == 1 ? ny : nz);
            real sn, cs;
            if constexpr (sizeof(real) == 8) sincos(kappa * d.r, &sn, &cs);
            else sincosf(kappa * d.r, &sn, &cs);
            const real dnx = ((al == 0 ? real(1) : real(0)) - na * nx) * ir;
            const real dny = ((al == 1 ? real(1) : real(0)) - na * ny) * ir;
            const real dnz = ((al == 2 ? real(1) : real(0)) - na * nz) * ir;
            const cplx<real> da{-sn * kappa * na, -(cs * kappa * na * nz + sn * dnz)};
            const cplx<real> db{cs * kappa * na * ny + sn * dny, -(cs * kappa * na * nx + sn * dnx)};
            // xi = Im(conj(a) da + b conj(db));  eta = conj(a) db - b conj(da)
            const real xi = (a.re * da.im - a.im * da.re) + (b.im * db.re - b.re * db.im);
            const cplx<real> eta{(a.re * db.re + a.im * db.im) - (b.re * da.re + b.im * da.im),
                                 (a.re * db.im - a.im * db.re) - (b.im * da.re - b.re * da.im)};
            const real phi = real(-2) * xi * Dim - (eta.re * Pre + eta.im * Pim) + (eta.re * Qre - eta.im * Qim);
            real dw = real(0);
            if (sp.switchflag) {
                if constexpr (sizeof(real) == 8) dw = -0.5 * sin(PI * d.r / rcut) * (PI / rcut) * na;
                else dw = -0.5f * sinf(float(PI) * d.r / rcut) * (float(PI) / rcut) * na;
            }
            dedr_out[s * 3 + al] = w * phi + dw * Sre;
        }
        __syncwarp();
    }
}

// Force on atom k of a system: F_k = sum_{j in N(k)} (dE_k/dr_kj - dE_j/dr_jk), neighbour lists
// sorted by index and symmetric; the slot of k in N(j) is found by binary search.
template <typename real>
__device__ __forceinline__ void gather_force(const int* __restrict__ nbr, const int* __restrict__ nnb,
                                             const real* __restrict__ dedr, int k, double F[3], int* status) {
    F[0] = F[1] = F[2] = 0.0;
    const int ck = nnb[k];
    const int* lk = nbr + (size_t)k * NMAX;
    const real* dk = dedr + (size_t)k * NMAX * 3;
    for (int s = 0; s < ck; ++s) {
        const int j = lk[s];
        const int cj = nnb[j];
        const int* lj = nbr + (size_t)j * NMAX;
        int lo = 0, hi = cj - 1, t = -1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int v = lj[mid];
            if (v == k) {
                t = mid;
                break;
            }
            if (v < k) lo = mid + 1;
            else hi = mid - 1;
        }
        const real* dj = dedr + ((size_t)j * NMAX + (t < 0 ? 0 : t)) * 3;
        if (t < 0) flag(status, ST_BADNEIGH);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double g = (double)dk[s * 3 + a];
            double h = t < 0 ? 0.0 : (double)dj[a];
            F[a] += g - h;
        }
    }
}

}  // namespace pmd
