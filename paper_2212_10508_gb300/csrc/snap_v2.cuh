// SNAP per-atom pass, second kernel design (one warp per atom, SIMT-uniform control flow).
//
//  U_tot and dE/dr passes: lane k handles neighbour k.  Each lane runs the whole half-layout
//  recursion of U(a_k, b_k) in registers with compile-time indices and coefficients (the
//  recursion of snap_device.cuh unrolled element by element, level by level, column by column).
//   * U pass: after each level the lanes' weighted values w_k U^j(g_k) are written to a padded
//     shared buffer and summed over the 32 lanes in a fixed order (deterministic), giving U_tot.
//   * dE/dr pass: each lane contracts its U(g_k) with four pre-weighted copies of Y (warp-wide
//     broadcast reads) and finishes dE_i/dr_ik for its own neighbour; no cross-lane work.
//  Y pass: the contraction jobs (output element, block) run in rounds in which every lane has a
//  job of the same sub-block size tb, each a uniform (tb+1) x (tb+1) loop (out-of-range rows and
//  columns get zero Clebsch-Gordan weight); every output belongs to one lane, which accumulates
//  it in shared memory in a fixed order.
#pragma once

#include "snap_device.cuh"

namespace pmd {

// ---- compile-time element metadata ------------------------------------------------------------
__host__ __device__ constexpr double csqrt(double x) {
    if (x <= 0.0) return 0.0;
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 200; ++i) {
        const double nr = 0.5 * (r + x / r);
        if (nr == r) break;
        r = nr;
    }
    return r;
}

// Traversal order: level tj, then column q ascending (m >= 0), then row p ascending.
struct HM {
    int tj, p, q;
    int pos;          // position within the level
    int nlev;         // elements in the level
    int hidx;         // row-major half index (Y half storage and job outputs)
    int src1, src2;   // traversal indices of the recursion sources (-1: zero coefficient)
    int yrule;        // 1: m = 0 column (b, conj a); 0: (a, -conj b)
    double c1, c2;    // coefficients of the U recursion (the kernels run the V recursion: 1, 1)
    double nrm;       // U = nrm * V, nrm = sqrt(p! (tj-p)! / (q! (tj-q)!))
    int full, mir, mirneg;
    double wD, wP, wQ, wS;
    int yp, ym;       // full indices of (p, q+1), (p, q-1) (-1: zero weight)
};

__host__ __device__ constexpr int trav(int tj, int p, int q) { return h_off(tj) + (q - h_qlo(tj)) * (tj + 1) + p; }

__host__ __device__ constexpr double cfact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

__host__ __device__ constexpr HM hm(int E) {
    HM m{};
    int tj = 0;
    while (E >= h_off(tj + 1)) ++tj;
    const int loc = E - h_off(tj);
    const int col = loc / (tj + 1), p = loc % (tj + 1), q = h_qlo(tj) + col;
    m.tj = tj;
    m.p = p;
    m.q = q;
    m.pos = loc;
    m.nlev = (tj + 1) * h_ncol(tj);
    m.hidx = h_off(tj) + p * h_ncol(tj) + col;
    m.src1 = m.src2 = -1;
    m.c1 = m.c2 = 0.0;
    m.yrule = 0;
    if (tj > 0) {
        if (2 * q > tj) {
            if (p >= 1) {
                m.src1 = trav(tj - 1, p - 1, q - 1);
                m.c1 = csqrt((double)p / q);
            }
            if (p <= tj - 1) {
                m.src2 = trav(tj - 1, p, q - 1);
                m.c2 = csqrt((double)(tj - p) / q);
            }
        } else {
            m.yrule = 1;
            if (p >= 1) {
                m.src1 = trav(tj - 1, p - 1, q);
                m.c1 = csqrt((double)p / (tj - q));
            }
            if (p <= tj - 1) {
                m.src2 = trav(tj - 1, p, q);
                m.c2 = csqrt((double)(tj - p) / (tj - q));
            }
        }
    }
    m.nrm = csqrt(cfact(p) * cfact(tj - p) / (cfact(q) * cfact(tj - q)));
    m.full = f_off(tj) + p * (tj + 1) + q;
    m.mir = 2 * q > tj ? f_off(tj) + (tj - p) * (tj + 1) + (tj - q) : -1;
    m.mirneg = ((p - q) & 1) != 0;
    const double w = 2 * q > tj ? 2.0 : 1.0;
    m.wD = w * (q - 0.5 * tj);
    m.wP = w * csqrt((double)(q + 1) * (tj - q));
    m.wQ = w * csqrt((double)(tj - q + 1) * q);
    m.wS = w;
    m.yp = q + 1 <= tj ? m.full + 1 : -1;
    m.ym = q - 1 >= 0 ? m.full - 1 : -1;
    if (m.wP == 0.0) m.yp = -1;
    if (m.wQ == 0.0) m.ym = -1;
    return m;
}

// f.apply<E>() for E = B, ..., N - 1 in increasing order (split in halves: nesting depth log2 N, so
// that the 652 elements of 2J = 14 stay within the compiler's instantiation depth).
template <int B, int N>
struct ForE {
    template <class F>
    __device__ __forceinline__ static void run(F& f) {
        if constexpr (N - B == 1) {
            f.template apply<B>();
        } else if constexpr (N - B > 1) {
            ForE<B, B + (N - B) / 2>::run(f);
            ForE<B + (N - B) / 2, N>::run(f);
        }
    }
};

// ---- per-lane recursion -------------------------------------------------------------------------
// The recursion runs on V^j_{pq} = U^j_{pq} / nrm_{pq} with nrm_{pq} = sqrt(p! (tj-p)! / (q! (tj-q)!))
// (p = j + m', q = j + m): the square-root coefficients of the U recursion are exactly absorbed, so
// V^j_{pq} = A1 V^{j-1/2}_{src1} + A2 V^{j-1/2}_{src2} with unit weights (V^0 = 1).  The sinks
// receive V; U = nrm V is applied once per atom (to the lane sums of U_tot, and folded into the
// weighted copies of Y that the dE/dr pass contracts with V).
template <typename real, int TJ, class Sink>
struct URec {
    cplx<real> u[Dims<TJ>::NHALF];
    cplx<real> a, b, ca, mcb;
    Sink& sink;
    __device__ __forceinline__ URec(cplx<real> a_, cplx<real> b_, Sink& s) : a(a_), b(b_), sink(s) {
        ca = {a.re, -a.im};
        mcb = {-b.re, b.im};
    }
    template <int E>
    __device__ __forceinline__ void apply() {
        constexpr HM m = hm(E);
        if constexpr (m.tj == 0) {
            u[E] = {real(1), real(0)};
        } else {
            const cplx<real> A1 = m.yrule ? b : a;
            const cplx<real> A2 = m.yrule ? ca : mcb;
            cplx<real> v{real(0), real(0)};
            if constexpr (m.src1 >= 0) v = cmul(A1, u[m.src1 >= 0 ? m.src1 : 0]);
            if constexpr (m.src2 >= 0) {
                const cplx<real> x = u[m.src2 >= 0 ? m.src2 : 0];
                v.re += A2.re * x.re - A2.im * x.im;
                v.im += A2.re * x.im + A2.im * x.re;
            }
            u[E] = v;
        }
        sink.template take<E>(u[E]);
    }
};

// per-element data used by lane-strided runtime loops (one table per CTA, in shared memory)
// ypH / ymH: half (row-major) index holding Y(p, q+1) / Y(p, q-1), -1 when the weight is zero;
// ymMode: 0 when Y(p, q-1) is stored directly, +-1 when it is the mirror image
// Y(p, q-1) = ymMode * conj(Y(tj-p, tj-q+1)) of a stored element.
template <typename real>
struct ElemRT {
    int full, mir, hidx, yp, ym, mirneg, diag;
    int ypH, ymH, ymMode;
    real wD, wP, wQ, wS;
    real nrm;   // U = nrm * V of the recursion
};

template <typename real, int TJ>
__device__ inline void fill_elem_table(ElemRT<real>* tab) {
    for (int e = threadIdx.x; e < Dims<TJ>::NHALF; e += blockDim.x) {
        const HM m = hm(e);
        const int nc = h_ncol(m.tj), ql = h_qlo(m.tj);
        const int ypH = m.yp >= 0 ? m.hidx + 1 : -1;
        int ymH = -1, ymMode = 0;
        if (m.ym >= 0) {
            if (m.q - 1 >= ql) {
                ymH = m.hidx - 1;
            } else {
                ymH = h_off(m.tj) + (m.tj - m.p) * nc + (m.tj - m.q + 1 - ql);
                ymMode = ((m.p - m.q + 1) & 1) ? -1 : 1;
            }
        }
        tab[e] = ElemRT<real>{m.full, m.mir, m.hidx, m.yp, m.ym, m.mirneg, m.p == m.q ? 1 : 0, ypH, ymH, ymMode,
                              real(m.wD), real(m.wP), real(m.wQ), real(m.wS), real(m.nrm)};
    }
}

// per-warp shared memory of the second design
template <typename real, int TJ>
struct WarpScratch2 {
    int nbr[NMAX];
    Vec4<real> disp[NMAX];
    cplx<real> full[Dims<TJ>::NFULL];                      // U_tot, then Y
    union {
        cplx<real> lv[16 * 33];                            // lane values of 16 elements (U pass)
        cplx<real> yh[Dims<TJ>::NHALF + 1];                // Y half accumulators (Y pass), +1 dummy
        cplx<real> yw[4 * Dims<TJ>::NHALF];                // weighted Y copies (dE/dr pass)
    };
};

// U pass sink: store w * U(g_k) of this lane; every 16 elements (traversal order) sum the
// stored values over the 32 lanes in a fixed order and add them to U_tot.
template <typename real, int TJ>
struct SinkU {
    WarpScratch2<real, TJ>& ws;
    const ElemRT<real>* tab;
    int lane;
    real w;
    bool first;
    template <int E>
    __device__ __forceinline__ void take(cplx<real> v) {
        constexpr int NH = Dims<TJ>::NHALF;
        ws.lv[(E & 15) * 33 + lane] = {w * v.re, w * v.im};
        if constexpr ((E & 15) == 15 || E == NH - 1) {
            constexpr int base = E & ~15;
            constexpr int cnt = E - base + 1;
            __syncwarp();
            if (lane < cnt) {
                real sr = 0, si = 0;
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const cplx<real> x = ws.lv[lane * 33 + j];
                    sr += x.re;
                    si += x.im;
                }
                // element base + lane in traversal order; identity on the diagonal (self term)
                const ElemRT<real>& t = tab[base + lane];
                const int f = t.full;
                sr *= t.nrm;   // V -> U
                si *= t.nrm;
                if (first) {
                    ws.full[f] = {sr + (t.diag ? real(1) : real(0)), si};
                } else {
                    ws.full[f].re += sr;
                    ws.full[f].im += si;
                }
            }
            __syncwarp();
        }
    }
};

// dE/dr pass sink: contraction of the lane's U(g_k) with the pre-weighted Y copies
template <typename real, int TJ>
struct SinkF {
    const cplx<real>* yw;   // [4][NHALF] in traversal order: wD*Y, wS*Y, wP*Y(q+1), wQ*Y(q-1)
    real Dim = 0, Sre = 0, Pre = 0, Pim = 0, Qre = 0, Qim = 0;
    template <int E>
    __device__ __forceinline__ void take(cplx<real> u) {
        constexpr HM m = hm(E);
        constexpr int NH = Dims<TJ>::NHALF;
        if constexpr (m.wD != 0.0) {
            const cplx<real> y = yw[E];
            Dim += y.re * u.im - y.im * u.re;
        }
        {
            const cplx<real> y = yw[NH + E];
            Sre += y.re * u.re + y.im * u.im;
        }
        if constexpr (m.yp >= 0) {
            const cplx<real> y = yw[2 * NH + E];
            Pre += y.re * u.re + y.im * u.im;
            Pim += y.re * u.im - y.im * u.re;
        }
        if constexpr (m.ym >= 0) {
            const cplx<real> y = yw[3 * NH + E];
            Qre += y.re * u.re + y.im * u.im;
            Qim += y.re * u.im - y.im * u.re;
        }
    }
};

struct NoSink {
    template <int E>
    __device__ __forceinline__ void take(const void*) {}
};

// ---- Y contraction in lockstep rounds ---------------------------------------------------------
// Job record (int4): x = out half index | blk << 16; y = (p1_0 + 32) | (q1_0 + 32) << 8 | ta << 16 | tb << 24;
// z = full offset of U^a | full offset of U^b << 16; w = CG offset of the block.
template <typename real, int TB>
__device__ __forceinline__ void y_job(const int4 J, const cplx<real>* __restrict__ U, const real* __restrict__ cg,
                                      const real* __restrict__ beff, cplx<real>* __restrict__ yh) {
    const int e = J.x & 0xffff, blk = J.x >> 16;
    const int p10 = (J.y & 0xff) - 32, q10 = ((J.y >> 8) & 0xff) - 32, ta = (J.y >> 16) & 0xff;
    const int ua = J.z & 0xffff, ub = J.z >> 16;
    const real* c = cg + J.w;
    real c2[TB + 1];
    int qc[TB + 1];
#pragma unroll
    for (int k = 0; k <= TB; ++k) {
        const int q1 = q10 + k;
        const bool ok = q1 >= 0 && q1 <= ta;
        qc[k] = ok ? q1 : 0;
        c2[k] = ok ? c[q1 * (TB + 1) + (TB - k)] : real(0);
    }
    real zr = 0, zi = 0;
#pragma unroll
    for (int i = 0; i <= TB; ++i) {
        const int p1 = p10 + i;
        const bool ok = p1 >= 0 && p1 <= ta;
        const real c1 = ok ? c[(ok ? p1 : 0) * (TB + 1) + (TB - i)] : real(0);
        const cplx<real>* Ua = U + ua + (ok ? p1 : 0) * (ta + 1);
        const cplx<real>* Ub = U + ub + (TB - i) * (TB + 1);
        real tr = 0, ti = 0;
#pragma unroll
        for (int k = 0; k <= TB; ++k) {
            const cplx<real> x = Ua[qc[k]];
            const cplx<real> y = Ub[TB - k];
            const real pr = x.re * y.re - x.im * y.im;
            const real pi = x.re * y.im + x.im * y.re;
            tr += c2[k] * pr;
            ti += c2[k] * pi;
        }
        zr += c1 * tr;
        zi += c1 * ti;
    }
    const real be = beff[blk];
    yh[e].re += be * zr;
    yh[e].im += be * zi;
}

template <typename real, int TJ>
__device__ __noinline__ void y_rounds(const int4* __restrict__ jobs, const unsigned char* __restrict__ round_tb,
                                         int nrounds, int lane, const cplx<real>* U, const real* cg, const real* beff,
                                         cplx<real>* yh) {
    for (int r = 0; r < nrounds; ++r) {
        const int4 J = jobs[r * 32 + lane];
        switch (round_tb[r]) {
#define PMD_YR_CASE(TB_) \
    case TB_:            \
        if constexpr (TB_ <= TJ) y_job<real, TB_>(J, U, cg, beff, yh); \
        break;
            PMD_YR_CASE(0) PMD_YR_CASE(1) PMD_YR_CASE(2) PMD_YR_CASE(3) PMD_YR_CASE(4) PMD_YR_CASE(5)
            PMD_YR_CASE(6) PMD_YR_CASE(7) PMD_YR_CASE(8) PMD_YR_CASE(9) PMD_YR_CASE(10) PMD_YR_CASE(11)
            PMD_YR_CASE(12) PMD_YR_CASE(13) PMD_YR_CASE(14)
#undef PMD_YR_CASE
            default: break;
        }
    }
}

// ---- mirror / expansion helpers (lane-strided loops over the element table) -------------------
template <typename real, int TJ>
__device__ __forceinline__ void mirror_full(cplx<real>* full, const ElemRT<real>* tab, int lane) {
    for (int e = lane; e < Dims<TJ>::NHALF; e += 32) {
        const ElemRT<real>& t = tab[e];
        if (t.mir >= 0) {
            const cplx<real> v = full[t.full];
            const real sg = t.mirneg ? real(-1) : real(1);
            full[t.mir] = {sg * v.re, -sg * v.im};
        }
    }
}

template <typename real, int TJ>
__device__ __forceinline__ void expand_y(const cplx<real>* yh, cplx<real>* full, const ElemRT<real>* tab, int lane) {
    for (int e = lane; e < Dims<TJ>::NHALF; e += 32) {
        const ElemRT<real>& t = tab[e];
        const cplx<real> v = yh[t.hidx];
        full[t.full] = v;
        if (t.mir >= 0) {
            const real sg = t.mirneg ? real(-1) : real(1);
            full[t.mir] = {sg * v.re, -sg * v.im};
        }
    }
}

// yw[0..3][E] = wD Y, wS Y, wP Y(q+1), wQ Y(q-1) in traversal order
template <typename real, int TJ>
__device__ __forceinline__ void weight_y(const cplx<real>* full, cplx<real>* yw, const ElemRT<real>* tab, int lane) {
    constexpr int NH = Dims<TJ>::NHALF;
    for (int e = lane; e < NH; e += 32) {
        const ElemRT<real>& t = tab[e];
        const cplx<real> y0 = full[t.full];
        // weights times nrm: the dE/dr pass contracts with V = U / nrm
        const real wD = t.wD * t.nrm, wS = t.wS * t.nrm, wP = t.wP * t.nrm, wQ = t.wQ * t.nrm;
        yw[e] = {wD * y0.re, wD * y0.im};
        yw[NH + e] = {wS * y0.re, wS * y0.im};
        const cplx<real> yp = full[t.yp >= 0 ? t.yp : t.full];
        const cplx<real> ym = full[t.ym >= 0 ? t.ym : t.full];
        yw[2 * NH + e] = {wP * yp.re, wP * yp.im};
        yw[3 * NH + e] = {wQ * ym.re, wQ * ym.im};
    }
}

// ---- the per-atom pass -------------------------------------------------------------------------
struct SnapV2Tables {
    const int4* jobs;              // [nrounds][32]
    const unsigned char* round_tb; // [nrounds]
    int nrounds;
};

template <typename real>
__device__ __forceinline__ void dedr_lane(const Vec4<real>& d, real kappa, real rcut, int sw, const cplx<real>& a,
                                          const cplx<real>& b, real w, real Dim, real Sre, real Pre, real Pim,
                                          real Qre, real Qim, real out[3]) {
    const real ir = real(1) / d.r;
    const real nx = d.x * ir, ny = d.y * ir, nz = d.z * ir;
    real sn, cs;
    if constexpr (sizeof(real) == 8) sincos(kappa * d.r, &sn, &cs);
    else sincosf(kappa * d.r, &sn, &cs);
    real swd = real(0);
    if (sw) {
        if constexpr (sizeof(real) == 8) swd = -0.5 * sin(PI * d.r / rcut) * (PI / rcut);
        else swd = -0.5f * sinf(float(PI) * d.r / rcut) * (float(PI) / rcut);
    }
#pragma unroll
    for (int al = 0; al < 3; ++al) {
        const real na = al == 0 ? nx : (al == 1 ? ny : nz);
        const real dnx = ((al == 0 ? real(1) : real(0)) - na * nx) * ir;
        const real dny = ((al == 1 ? real(1) : real(0)) - na * ny) * ir;
        const real dnz = ((al == 2 ? real(1) : real(0)) - na * nz) * ir;
        const cplx<real> da{-sn * kappa * na, -(cs * kappa * na * nz + sn * dnz)};
        const cplx<real> db{cs * kappa * na * ny + sn * dny, -(cs * kappa * na * nx + sn * dnx)};
        const real xi = (a.re * da.im - a.im * da.re) + (b.im * db.re - b.re * db.im);
        const cplx<real> eta{(a.re * db.re + a.im * db.im) - (b.re * da.re + b.im * da.im),
                             (a.re * db.im - a.im * db.re) - (b.im * da.re - b.re * da.im)};
        const real phi = real(-2) * xi * Dim - (eta.re * Pre + eta.im * Pim) + (eta.re * Qre - eta.im * Qim);
        out[al] = w * phi + swd * na * Sre;
    }
}

// One round of 32 neighbours of the U pass (kept out of line so that the recursion's
// element array is scalarised into registers).
template <typename real, int TJ>
__device__ __noinline__ void u_pass_round(WarpScratch2<real, TJ>& ws, const ElemRT<real>* tab, int lane, int k,
                                          int cnt, real kappa, real rcut, int sw, bool first) {
    cplx<real> a{real(1), real(0)}, b{real(0), real(0)};
    real w = real(0);
    if (k < cnt) cayley_klein<real>(ws.disp[k], kappa, rcut, sw, a, b, w);
    SinkU<real, TJ> sink{ws, tab, lane, w, first};
    URec<real, TJ, SinkU<real, TJ>> rec(a, b, sink);
    ForE<0, Dims<TJ>::NHALF>::run(rec);
}

// One round of 32 neighbours of the dE/dr pass.
template <typename real, int TJ>
__device__ __noinline__ void f_pass_round(WarpScratch2<real, TJ>& ws, int k, int cnt, real kappa, real rcut, int sw,
                                          real* dedr_out) {
    cplx<real> a{real(1), real(0)}, b{real(0), real(0)};
    real w = real(0);
    const Vec4<real> d = ws.disp[k < cnt ? k : 0];
    if (k < cnt) cayley_klein<real>(d, kappa, rcut, sw, a, b, w);
    SinkF<real, TJ> sink{ws.yw};
    URec<real, TJ, SinkF<real, TJ>> rec(a, b, sink);
    ForE<0, Dims<TJ>::NHALF>::run(rec);
    if (k < cnt) {
        real out[3];
        dedr_lane<real>(d, kappa, rcut, sw, a, b, w, sink.Dim, sink.Sre, sink.Pre, sink.Pim, sink.Qre, sink.Qim, out);
        dedr_out[k * 3 + 0] = out[0];
        dedr_out[k * 3 + 1] = out[1];
        dedr_out[k * 3 + 2] = out[2];
    }
}

template <typename real, int TJ>
__device__ __noinline__ void snap_atom_warp2(WarpScratch2<real, TJ>& ws, const ElemRT<real>* tab, const SnapV2Tables& yt,
                                const real* __restrict__ cg,
                                const real* __restrict__ beff, const SnapDevParams& sp, int lane, int n, int i,
                                const double* q64, const float4* qf, const double box[3], int* nbr_out,
                                int* nnb_out, real* dedr_out, cplx<real>* utot_out, int* status,
                                bool want_forces = true) {
    constexpr int NH = Dims<TJ>::NHALF;
    const real kappa = real(sp.rfac0 * PI / sp.rcut);
    const real rcut = real(sp.rcut);
    const int cnt = warp_neighbors<real>(ws.nbr, ws.disp, lane, n, i, q64, qf, box, sp.rcut, status);
    for (int s = lane; s < cnt; s += 32) nbr_out[s] = ws.nbr[s];
    if (lane == 0) *nnb_out = cnt;
    const int nround = (cnt + 31) / 32;

    // U_tot = I + sum_k w_k U(g_k): lane = neighbour, fixed-order sums over lanes
    for (int r = 0; r < (nround > 0 ? nround : 1); ++r)
        u_pass_round<real, TJ>(ws, tab, lane, r * 32 + lane, cnt, kappa, rcut, sp.switchflag, r == 0);
    mirror_full<real, TJ>(ws.full, tab, lane);
    __syncwarp();
    if (utot_out) {
        for (int e = lane; e < Dims<TJ>::NFULL; e += 32) utot_out[e] = ws.full[e];
    }
    if (!want_forces) {   // energies only: the adjoint and force passes are not needed
        __syncwarp();
        return;
    }

    // Y = sum_blocks beta_eff Z (lockstep rounds, lane-owned outputs)
    for (int e = lane; e <= NH; e += 32) ws.yh[e] = {real(0), real(0)};
    __syncwarp();
    y_rounds<real, TJ>(yt.jobs, yt.round_tb, yt.nrounds, lane, ws.full, cg, beff, ws.yh);
    __syncwarp();
    expand_y<real, TJ>(ws.yh, ws.full, tab, lane);
    __syncwarp();
    weight_y<real, TJ>(ws.full, ws.yw, tab, lane);
    __syncwarp();

    // dE_i/dr_ik: lane = neighbour
    for (int r = 0; r < nround; ++r)
        f_pass_round<real, TJ>(ws, r * 32 + lane, cnt, kappa, rcut, sp.switchflag, dedr_out);
    __syncwarp();
}

}  // namespace pmd
