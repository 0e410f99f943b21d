// SNAP per-atom pass, batched design (FP32): a CTA of SB_WARPS warps evaluates SB_ATOMS = 32
// atoms at a time in three phases separated by CTA barriers.
//
//  U phase : warp per atom, lane = neighbour; each lane runs the unrolled half-layout recursion
//            of U(a_k, b_k) (snap_v2.cuh) and the lanes' weighted values are summed over the 32
//            lanes in a fixed order.  U_tot of the batch is kept in shared memory as
//            [element][atom] with a padded leading dimension (SB_LD = 33).
//  Y phase : lane = atom.  Y^J = sum_blocks beta_eff(J,a,b) Z^J_{ab} on the half layout, in
//            stages of sub-block sizes b (CTA barrier in between: few variants of unrolled code
//            at a time).  In a stage warps take whole output rows (J, m') from a shared counter
//            and run, per block, the Clebsch-Gordan double sum of the row's outputs: for each row m1' of U^a, the window of U^a columns that
//            the row's outputs share and one row of U^b are loaded once into registers and
//            reused by all outputs.  Loop bounds skip out-of-range terms, all control flow and
//            index arithmetic is warp-uniform, and every lane reads its own atom's element
//            (stride-1 across lanes: no bank conflicts).
//  dE/dr   : warp per atom, lane = neighbour: each lane contracts its U(g_k) with three
//            pre-weighted copies of the atom's Y and finishes dE_i/dr_ik.
// Every sum runs in a fixed order (no atomics): results are bitwise reproducible.
#pragma once

#include "snap_v2.cuh"

namespace pmd {

constexpr int SB_ATOMS = 32;              // atoms per batch = lanes of the Y phase
constexpr int SB_LD = 33;                 // leading dimension of the [element][atom] arrays
constexpr int SB_WARPS = 16;             // warps per CTA (at most; the fine kernel also runs with 8)
constexpr int SB_THREADS = SB_WARPS * 32;
constexpr int SB_CHUNK = 8;               // U-pass elements summed per lane-sum round (4 lanes each)
constexpr int SB_SMALL_TB = 3;            // sub-block sizes tb <= this share one Y stage
constexpr int SB_MAX_STAGES = 16;
constexpr int SB_GUARD = 16;              // zero rows before and after U_tot (>= twojmax)

// Y stages: tb <= SB_SMALL_TB together, then one per larger tb
__host__ __device__ constexpr int sb_stage_of(int tb) { return tb <= SB_SMALL_TB ? 0 : tb - SB_SMALL_TB; }
__host__ __device__ constexpr int sb_num_stages(int twojmax) { return sb_stage_of(twojmax) + 1; }

// Shared memory of one CTA.  Aliases: the U-pass lane buffers live in the Y array (unused
// during the U phase), the weighted Y copies of the dE/dr phase in the U array (unused after
// the Y phase).
template <int TJ>
struct SBShared {
    float* beff;               // beta_eff per block
    ElemRT<float>* tab;        // element table (traversal order)
    float2* ut;                // [NFULL][SB_LD] U_tot of the batch
    float2* yt;                // [NHALF][SB_LD] Y of the batch (row-major half index)
    int* nbr;                  // [SB_ATOMS][NMAX]
    int* nnb;                  // [SB_ATOMS]
    int* ctr;                  // [SB_MAX_STAGES] row counters of the Y stages
    Vec4<float>* disp;         // [SB_ATOMS][NMAX]
    __device__ float2* lv(int warp) const { return yt + warp * SB_CHUNK * SB_LD; }
    __device__ float2* yw(int warp) const { return ut + warp * 3 * Dims<TJ>::NHALF; }
};

// U_tot region: SB_GUARD zero rows, NFULL rows, SB_GUARD zero rows.  The Y phase reads whole
// column windows of U^a rows; slots outside the row (zero weight) read a neighbouring row or a
// guard row, never outside the region.  The weighted Y copies of the dE/dr phase alias the NFULL
// rows only, so the guards stay zero.
template <int TJ>
__host__ __device__ constexpr size_t sb_ut_elems() {
    static_assert((size_t)SB_WARPS * 3 * Dims<TJ>::NHALF <= (size_t)Dims<TJ>::NFULL * SB_LD, "yw alias");
    static_assert(SB_GUARD >= TJ, "guard rows");
    return (size_t)(Dims<TJ>::NFULL + 2 * SB_GUARD) * SB_LD;
}
template <int TJ>
__host__ __device__ constexpr size_t sb_yt_elems() {
    const size_t a = (size_t)Dims<TJ>::NHALF * SB_LD, b = (size_t)SB_WARPS * SB_CHUNK * SB_LD;
    return a > b ? a : b;
}

// Extra work for idle FP64 pipes: called once per batch by every warp of the CTA at the start of
// the largest Y stage, before the warp takes rows (the row counter balances the stage).
struct SBNoSide {
    __device__ void operator()(int, int) const {}
};

// Run-time shape of the batched pass (chosen by pmd_engine_autotune; defaults below).
struct SBShape {
    int rows2_atoms = 16;   // batches of at most this many atoms (<= 16) run the Y phase 2 rows per warp
    int rows4_atoms = 8;    // ... and of at most this many atoms (<= 8) 4 rows per warp
    int noise_stage = -1;   // Y stage that also draws the Gaussian increments (-1: the stage of b = 6)
};

// Device tables of the batched Y contraction.
struct SBTables {
    const int4* jobs;     // job records
    const int2* rows;     // job range of each (stage, row)
    const int* sptr;      // row ranges of the stages
    const float* coef;    // per-job Clebsch-Gordan weights
    const int2* groups;   // (first row, count) groups of equal-width rows
    const int* gptr;      // [2][nstages][2] group ranges [begin, end) per stage, for 2 and 4 rows per warp pass
};

// ---- U phase -----------------------------------------------------------------------------------
// Sink of the U recursion: store w * U(g_k) of this lane; every SB_CHUNK elements (traversal
// order) sum the stored values over the 32 lanes in a fixed order (per element: four partial
// sums of 8 lanes, combined pairwise) and add them to U_tot.
static_assert(SB_CHUNK == 8, "the lane sums map 8 elements x 4 quarters onto 32 lanes");

template <int TJ>
struct SinkUB {
    float2* lv;
    float2* ut;
    const ElemRT<float>* tab;
    int lane, slot;
    float w;
    bool first;
    template <int E>
    __device__ __forceinline__ void take(cplx<float> v) {
        constexpr int NH = Dims<TJ>::NHALF;
        lv[(E % SB_CHUNK) * SB_LD + lane] = make_float2(w * v.re, w * v.im);
        if constexpr ((E % SB_CHUNK) == SB_CHUNK - 1 || E == NH - 1) {
            constexpr int base = E - E % SB_CHUNK;
            constexpr int cnt = E - base + 1;
            __syncwarp();
            // all 32 lanes: lane (e = lane & 7, quarter h = lane >> 3) sums neighbour lanes
            // 8h..8h+7 of element e; the four quarters are combined by two xor-shuffles
            const int e = lane & 7, h = lane >> 3;
            float sr = 0.f, si = 0.f;
            if (e < cnt) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float2 x = lv[e * SB_LD + 8 * h + j];
                    sr += x.x;
                    si += x.y;
                }
            }
            sr += __shfl_xor_sync(0xffffffffu, sr, 8);
            si += __shfl_xor_sync(0xffffffffu, si, 8);
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            if (h == 0 && e < cnt) {
                // element base + e in traversal order; identity on the diagonal (self term)
                const ElemRT<float>& t = tab[base + e];
                float2* d = ut + t.full * SB_LD + slot;
                sr *= t.nrm;   // V -> U
                si *= t.nrm;
                if (first) {
                    *d = make_float2(sr + (t.diag ? 1.f : 0.f), si);
                } else {
                    const float2 o = *d;
                    *d = make_float2(o.x + sr, o.y + si);
                }
            }
            __syncwarp();
        }
    }
};

template <int TJ>
__device__ __noinline__ void sb_u_round(float2* lv, float2* ut, const Vec4<float>* disp, const ElemRT<float>* tab,
                                        int lane, int slot, int k, int cnt, float kappa, float rcut, int sw,
                                        bool first) {
    cplx<float> a{1.f, 0.f}, b{0.f, 0.f};
    float w = 0.f;
    if (k < cnt) cayley_klein<float>(disp[k], kappa, rcut, sw, a, b, w);
    SinkUB<TJ> sink{lv, ut, tab, lane, slot, w, first};
    URec<float, TJ, SinkUB<TJ>> rec(a, b, sink);
    ForE<0, Dims<TJ>::NHALF>::run(rec);
}

// ---- Y phase -----------------------------------------------------------------------------------
// One job: output row (tj, p) of the half layout (NC = h_ncol(tj) outputs, columns q = qlo..tj)
// and one block (ta, tb = TB, J = tj), s = (ta + tb - tj)/2.  Output (p, q) sums over rows
// p1 = p + s - TB + i of U^a (i = 0..TB, p2 = TB - i) and columns q1 = q + s - TB + k of U^a
// (k = 0..TB, q2 = TB - k):  C(p1, p2) C(q1, q2) U^a[p1][q1] U^b[p2][q2].  With the window
// slot w = q1 - (qlo + s - TB), output o = q - qlo uses slot w = o + k.  All TB + NC slots are
// read (no per-slot test): out-of-range columns carry zero weight.  Arithmetic on FP32 pairs
// (sm_100+ paired FMA): per term cx = c2 (xr, xi), S += cx * (yr, yi), T += cx * (yi, yr), so
// that S = (sum c xr yr, sum c xi yi) and T = (sum c xr yi, sum c xi yr); each row's S and T are
// scaled by its weight c1 and Z = (S.x - S.y, T.x + T.y) is formed once per job.
// Job record: x = ta | tb << 4 | tj << 8 | p << 12 | ilo << 16 | ihi << 20 | o0 << 24 (rows i
// visited: all valid rows, or in a diagonal block ta = tb only i <= i* = tb - p10 - i with the rows
// i < i* weighted twice, since rows i and i* sum to the same value; o0 = 1: the row's outputs start
// at column qlo + 1, the middle column being filled from its mirror image); y = offset of the job's
// weights in coef
// (column weights c2[o][k], zero where q1 is out of range, then row weights c1[i]);
// z = full offset of U^a | full offset of U^b << 16; w = half index of (tj, p, qlo) | blk << 16.
template <int TB, int NC>
__device__ __forceinline__ void sb_yjob(const int4 J, const float2* __restrict__ ut, const float* __restrict__ coef,
                                        const float* __restrict__ beff, float2* __restrict__ yt, int lane) {
    const int ta = J.x & 15, tj = (J.x >> 8) & 15, p = (J.x >> 12) & 15;
    const int s = (ta + TB - tj) >> 1;
    const int p10 = p + s - TB;
    const int c0 = ((tj + 1) >> 1) + ((J.x >> 24) & 1) + s - TB;   // first output column qlo + o0
    constexpr int N2 = NC * (TB + 1), NV = (N2 + 3) / 4;
    float c2[NV * 4];
    const float4* cp = reinterpret_cast<const float4*>(coef + J.y);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float4 t = __ldg(cp + v);
        c2[4 * v] = t.x;
        c2[4 * v + 1] = t.y;
        c2[4 * v + 2] = t.z;
        c2[4 * v + 3] = t.w;
    }
    const float* c1p = coef + J.y + N2;
    const int ilo = (J.x >> 16) & 15, ihi = (J.x >> 20) & 15;   // rows visited (host: job_rows)
    const int ua = J.z & 0xffff, ub = J.z >> 16;
    // paired accumulators: zS = sum c1 c2 (xr yr, xi yi), zT = sum c1 c2 (xr yi, xi yr)
    float2 zS[NC], zT[NC];
#pragma unroll
    for (int o = 0; o < NC; ++o) zS[o] = zT[o] = make_float2(0.f, 0.f);
    for (int i = ilo; i <= ihi; ++i) {
        const int p1 = p10 + i;
        const float c1 = __ldg(c1p + i);
        const float2* yb = ut + (ub + (TB - i) * (TB + 1)) * SB_LD + lane;
        float2 y[TB + 1], ys[TB + 1];
#pragma unroll
        for (int k = 0; k <= TB; ++k) {
            y[k] = yb[(TB - k) * SB_LD];
            ys[k] = make_float2(y[k].y, y[k].x);
        }
        const float2* xb = ut + (ua + p1 * (ta + 1) + c0) * SB_LD + lane;
        float2 S[NC], T[NC];
#pragma unroll
        for (int o = 0; o < NC; ++o) S[o] = T[o] = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < TB + NC; ++w) {
            const float2 x = xb[w * SB_LD];
#pragma unroll
            for (int o = 0; o < NC; ++o) {
                const int k = w - o;
                if (k < 0 || k > TB) continue;
                const float cc = c2[o * (TB + 1) + k];
                const float2 cx = __fmul2_rn(make_float2(cc, cc), x);
                S[o] = __ffma2_rn(cx, y[k], S[o]);
                T[o] = __ffma2_rn(cx, ys[k], T[o]);
            }
        }
        const float2 cc1 = make_float2(c1, c1);
#pragma unroll
        for (int o = 0; o < NC; ++o) {
            zS[o] = __ffma2_rn(cc1, S[o], zS[o]);
            zT[o] = __ffma2_rn(cc1, T[o], zT[o]);
        }
    }
    const float be = beff[J.w >> 16];
    float2* out = yt + (J.w & 0xffff) * SB_LD + lane;
#pragma unroll
    for (int o = 0; o < NC; ++o) {
        const float zr = zS[o].x - zS[o].y, zi = zT[o].x + zT[o].y;
        const float2 v = out[o * SB_LD];
        out[o * SB_LD] = make_float2(v.x + be * zr, v.y + be * zi);
    }
}

// The same contraction for a warp whose sub-warps of 32/R lanes each run a job of a different row
// (few atoms: lane la = lane % (32/R) of sub-warp lane / (32/R) is atom la).  The job parameters
// are per lane; all sub-warps run the same (TB, NC) variant, the row loop covers the union of the
// sub-warps' row ranges, and a lane outside its own range reads row 0 (clamped) with zero weight.
// Each output receives exactly the operations of the one-row form, in the same order.
template <int TB, int NC>
__device__ __forceinline__ void sb_yjob_m(const int4 J, bool valid, const float2* __restrict__ ut,
                                          const float* __restrict__ coef, const float* __restrict__ beff,
                                          float2* __restrict__ yt, int la) {
    const int ta = J.x & 15, tj = (J.x >> 8) & 15, p = (J.x >> 12) & 15;
    const int ilo = valid ? (J.x >> 16) & 15 : TB + 1, ihi = valid ? (J.x >> 20) & 15 : -1;
    const int s = (ta + TB - tj) >> 1;
    const int p10 = p + s - TB;
    const int c0 = ((tj + 1) >> 1) + ((J.x >> 24) & 1) + s - TB;
    constexpr int N2 = NC * (TB + 1), NV = (N2 + 3) / 4;
    float c2[NV * 4];
    const float4* cp = reinterpret_cast<const float4*>(coef + (valid ? J.y : 0));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float4 t = __ldg(cp + v);
        c2[4 * v] = t.x;
        c2[4 * v + 1] = t.y;
        c2[4 * v + 2] = t.z;
        c2[4 * v + 3] = t.w;
    }
    const float* c1p = coef + (valid ? J.y : 0) + N2;
    const int wlo = __reduce_min_sync(0xffffffffu, ilo), whi = __reduce_max_sync(0xffffffffu, ihi);
    const int ua = J.z & 0xffff, ub = J.z >> 16;
    float2 zS[NC], zT[NC];
#pragma unroll
    for (int o = 0; o < NC; ++o) zS[o] = zT[o] = make_float2(0.f, 0.f);
    for (int i = wlo; i <= whi; ++i) {
        const bool on = i >= ilo && i <= ihi;
        const int p1 = on ? p10 + i : 0;
        const float c1 = on ? __ldg(c1p + i) : 0.f;
        const float2* yb = ut + (ub + (TB - i) * (TB + 1)) * SB_LD + la;
        float2 y[TB + 1], ys[TB + 1];
#pragma unroll
        for (int k = 0; k <= TB; ++k) {
            y[k] = yb[(TB - k) * SB_LD];
            ys[k] = make_float2(y[k].y, y[k].x);
        }
        const float2* xb = ut + (ua + p1 * (ta + 1) + c0) * SB_LD + la;
        float2 S[NC], T[NC];
#pragma unroll
        for (int o = 0; o < NC; ++o) S[o] = T[o] = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < TB + NC; ++w) {
            const float2 x = xb[w * SB_LD];
#pragma unroll
            for (int o = 0; o < NC; ++o) {
                const int k = w - o;
                if (k < 0 || k > TB) continue;
                const float cc = c2[o * (TB + 1) + k];
                const float2 cx = __fmul2_rn(make_float2(cc, cc), x);
                S[o] = __ffma2_rn(cx, y[k], S[o]);
                T[o] = __ffma2_rn(cx, ys[k], T[o]);
            }
        }
        if (on) {
            const float2 cc1 = make_float2(c1, c1);
#pragma unroll
            for (int o = 0; o < NC; ++o) {
                zS[o] = __ffma2_rn(cc1, S[o], zS[o]);
                zT[o] = __ffma2_rn(cc1, T[o], zT[o]);
            }
        }
    }
    if (valid) {
        const float be = beff[J.w >> 16];
        float2* out = yt + (J.w & 0xffff) * SB_LD + la;
#pragma unroll
        for (int o = 0; o < NC; ++o) {
            const float zr = zS[o].x - zS[o].y, zi = zT[o].x + zT[o].y;
            const float2 v = out[o * SB_LD];
            out[o * SB_LD] = make_float2(v.x + be * zr, v.y + be * zi);
        }
    }
}

// One warp pass over a group of cnt <= R rows of equal width and one sub-block size TB (a stage
// b >= 4): sub-warp r runs the jobs of row first + r, in order.
template <int TJ>
__device__ __noinline__ void sb_y_group(const SBTables tb, int2 G, int R, const float2* ut, const float* beff,
                                        float2* yt, int lane) {
    const int per = 32 / R, sub = lane / per, la = lane - sub * per;
    const bool have = sub < G.y;
    const int2 rj = have ? tb.rows[G.x + sub] : make_int2(0, 0);
    const int len = rj.y - rj.x;
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    const int4 J0 = tb.jobs[tb.rows[G.x].x];   // sub-warp 0's first job fixes the variant
    const int tbs = (J0.x >> 4) & 15, tj0 = (J0.x >> 8) & 15;
    const int nc = tj0 + 1 - ((tj0 + 1) >> 1) - ((J0.x >> 24) & 1);
    for (int t = 0; t < maxlen; ++t) {
        const bool valid = have && t < len;
        const int4 J = valid ? tb.jobs[rj.x + t] : J0;
        switch (nc * 16 + tbs) {
#define PMD_SBM_CASE(NC_, TB_)                                                                             \
    case NC_ * 16 + TB_:                                                                                   \
        if constexpr (TB_ <= TJ && NC_ <= h_ncol(TJ)) sb_yjob_m<TB_, NC_>(J, valid, ut, tb.coef, beff, yt, la); \
        break;
#define PMD_SBM_ROW(NC_) PMD_SBM_CASE(NC_, 4) PMD_SBM_CASE(NC_, 5) PMD_SBM_CASE(NC_, 6) PMD_SBM_CASE(NC_, 7) PMD_SBM_CASE(NC_, 8)
            PMD_SBM_ROW(1)
            PMD_SBM_ROW(2)
            PMD_SBM_ROW(3)
            PMD_SBM_ROW(4)
            PMD_SBM_ROW(5)
#undef PMD_SBM_ROW
#undef PMD_SBM_CASE
            default: break;
        }
    }
}

// Jobs [j0, j1) of one row, in order.
template <int TJ>
__device__ __noinline__ void sb_y_row(const int4* __restrict__ jobs, int j0, int j1, const float2* ut,
                                      const float* coef, const float* beff, float2* yt, int lane) {
    for (int j = j0; j < j1; ++j) {
        const int4 J = jobs[j];
        const int tb = (J.x >> 4) & 15, tj = (J.x >> 8) & 15;
        const int nc = tj + 1 - ((tj + 1) >> 1) - ((J.x >> 24) & 1);
        switch (nc * 16 + tb) {
#define PMD_SB_CASE(NC_, TB_)                                                         \
    case NC_ * 16 + TB_:                                                              \
        if constexpr (TB_ <= TJ && NC_ <= h_ncol(TJ)) sb_yjob<TB_, NC_>(J, ut, coef, beff, yt, lane); \
        break;
#define PMD_SB_ROW(NC_)                                                                          \
    PMD_SB_CASE(NC_, 0) PMD_SB_CASE(NC_, 1) PMD_SB_CASE(NC_, 2) PMD_SB_CASE(NC_, 3)              \
    PMD_SB_CASE(NC_, 4) PMD_SB_CASE(NC_, 5) PMD_SB_CASE(NC_, 6) PMD_SB_CASE(NC_, 7) PMD_SB_CASE(NC_, 8)
            PMD_SB_ROW(1)
            PMD_SB_ROW(2)
            PMD_SB_ROW(3)
            PMD_SB_ROW(4)
            PMD_SB_ROW(5)
#undef PMD_SB_ROW
#undef PMD_SB_CASE
            default: break;
        }
    }
}

// The whole Y phase of a batch (all threads of the CTA; ends with a CTA barrier).
template <int TJ, class Side = SBNoSide>
__device__ __forceinline__ void sb_y_phase(const SBShared<TJ>& sh, const SBTables& tb, int lane, int na = SB_ATOMS,
                                           const Side& side = Side(), const SBShape& shape = SBShape()) {
    const int side_stage = shape.noise_stage >= 0 && shape.noise_stage < sb_num_stages(TJ)
                               ? shape.noise_stage : sb_stage_of(TJ >= 6 ? 6 : TJ);
    constexpr int NST = sb_num_stages(TJ);
    const int2* __restrict__ rows = tb.rows;
    const int* __restrict__ sptr = tb.sptr;
    // rows per warp pass: 4 sub-warps of 8 lanes for <= 8 atoms, 2 of 16 for <= 16 (stages b >= 4)
    const int R = na <= shape.rows4_atoms && na <= 8 ? 4 : (na <= shape.rows2_atoms && na <= 16 ? 2 : 1);
    for (int x = threadIdx.x; x < Dims<TJ>::NHALF * SB_LD; x += blockDim.x) sh.yt[x] = make_float2(0.f, 0.f);
    if (threadIdx.x < SB_MAX_STAGES) sh.ctr[threadIdx.x] = 0;
    __syncthreads();
    for (int st = 0; st < sb_num_stages(TJ); ++st) {   // stages of sub-block sizes
        const int r0 = sptr[st], r1 = sptr[st + 1];
        if (st == side_stage) side(threadIdx.x >> 5, lane);
        if (r0 == r1) continue;
        if (R > 1 && st > 0) {   // multi-row warps over the stage's row groups
            const int* gp = tb.gptr + ((R == 2 ? 0 : NST) + st) * 2;   // [begin, end) of the stage's groups
            const int g0 = gp[0], g1 = gp[1];
            for (;;) {
                int g = 0;
                if (lane == 0) g = atomicAdd(&sh.ctr[st], 1);
                g = g0 + __shfl_sync(0xffffffffu, g, 0);
                if (g >= g1) break;
                sb_y_group<TJ>(tb, tb.groups[g], R, sh.ut, sh.beff, sh.yt, lane);
            }
        } else {
            for (;;) {
                int r = 0;
                if (lane == 0) r = atomicAdd(&sh.ctr[st], 1);
                r = r0 + __shfl_sync(0xffffffffu, r, 0);
                if (r >= r1) break;
                const int2 Rw = rows[r];
                sb_y_row<TJ>(tb.jobs, Rw.x, Rw.y, sh.ut, tb.coef, sh.beff, sh.yt, lane);
            }
        }
        __syncthreads();
    }
}

// Middle column of integer J (q = J/2 in doubled units, m = 0): rows p > J/2 are not computed by
// the Y jobs; Y(p, q) = (-1)^(p-q) conj Y(tj - p, q).  All threads; ends with a CTA barrier.
template <int TJ>
__device__ __forceinline__ void sb_fill_middle(float2* yt) {
    constexpr int NFILL = (TJ / 2) * (TJ / 2 + 1) / 2;   // sum over even tj <= TJ of tj / 2
    for (int x = threadIdx.x; x < NFILL * SB_ATOMS; x += blockDim.x) {
        const int atom = x % SB_ATOMS;
        int f = x / SB_ATOMS, tj = 2;
        while (f >= tj / 2) {
            f -= tj / 2;
            tj += 2;
        }
        const int q = tj / 2, p = q + 1 + f;
        const int nc = tj + 1 - (tj + 1) / 2;
        const int dst = h_off(tj) + p * nc, src = h_off(tj) + (tj - p) * nc;   // column q = qlo: offset 0
        const float2 v = yt[src * SB_LD + atom];
        const float sg = ((p - q) & 1) ? -1.f : 1.f;
        yt[dst * SB_LD + atom] = make_float2(sg * v.x, -sg * v.y);
    }
    __syncthreads();
}

// ---- dE/dr phase -------------------------------------------------------------------------------
// yw[0..2][E] (traversal order) = wS Y(p,q), wP Y(p,q+1), wQ Y(p,q-1) of the atom in slot.
template <int TJ>
__device__ __forceinline__ void sb_weight_y(const float2* yt, int slot, float2* yw, const ElemRT<float>* tab,
                                            int lane) {
    constexpr int NH = Dims<TJ>::NHALF;
    for (int e = lane; e < NH; e += 32) {
        const ElemRT<float>& t = tab[e];
        const float2 y0 = yt[t.hidx * SB_LD + slot];
        float2 yp = make_float2(0.f, 0.f), ym = make_float2(0.f, 0.f);
        if (t.ypH >= 0) yp = yt[t.ypH * SB_LD + slot];
        if (t.ymH >= 0) {
            ym = yt[t.ymH * SB_LD + slot];
            if (t.ymMode != 0) ym = make_float2(t.ymMode * ym.x, -t.ymMode * ym.y);
        }
        // weights times nrm: the dE/dr pass contracts with V = U / nrm
        const float wS = t.wS * t.nrm, wP = t.wP * t.nrm, wQ = t.wQ * t.nrm;
        yw[e] = make_float2(wS * y0.x, wS * y0.y);
        yw[NH + e] = make_float2(wP * yp.x, wP * yp.y);
        yw[2 * NH + e] = make_float2(wQ * ym.x, wQ * ym.y);
    }
}

template <int TJ>
struct SinkFB {
    const float2* yw;
    float Dim = 0.f, Sre = 0.f, Pre = 0.f, Pim = 0.f, Qre = 0.f, Qim = 0.f;
    template <int E>
    __device__ __forceinline__ void take(cplx<float> u) {
        constexpr HM m = hm(E);
        constexpr int NH = Dims<TJ>::NHALF;
        const float2 y = yw[E];
        Sre += y.x * u.re + y.y * u.im;
        if constexpr (m.wD != 0.0) {
            constexpr float r = float(m.wD / m.wS);
            Dim += r * (y.x * u.im - y.y * u.re);
        }
        if constexpr (m.yp >= 0) {
            const float2 yp = yw[NH + E];
            Pre += yp.x * u.re + yp.y * u.im;
            Pim += yp.x * u.im - yp.y * u.re;
        }
        if constexpr (m.ym >= 0) {
            const float2 ym = yw[2 * NH + E];
            Qre += ym.x * u.re + ym.y * u.im;
            Qim += ym.x * u.im - ym.y * u.re;
        }
    }
};

template <int TJ>
__device__ __noinline__ void sb_f_round(const float2* yw, const Vec4<float>* disp, int k, int cnt, float kappa,
                                        float rcut, int sw, float* dedr_out) {
    cplx<float> a{1.f, 0.f}, b{0.f, 0.f};
    float w = 0.f;
    const Vec4<float> d = disp[k < cnt ? k : 0];
    if (k < cnt) cayley_klein<float>(d, kappa, rcut, sw, a, b, w);
    SinkFB<TJ> sink{yw};
    URec<float, TJ, SinkFB<TJ>> rec(a, b, sink);
    ForE<0, Dims<TJ>::NHALF>::run(rec);
    if (k < cnt) {
        float out[3];
        dedr_lane<float>(d, kappa, rcut, sw, a, b, w, sink.Dim, sink.Sre, sink.Pre, sink.Pim, sink.Qre, sink.Qim, out);
        dedr_out[k * 3 + 0] = out[0];
        dedr_out[k * 3 + 1] = out[1];
        dedr_out[k * 3 + 2] = out[2];
    }
}

// ---- one batch ---------------------------------------------------------------------------------
// Where atom `slot` of the batch lives and where its results go.
struct SBAtom {
    const double* q64;     // member positions [3][n]
    const float4* qf;      // member positions wrapped to FP32 [n]
    int i;                 // atom index in its member
    int* nbr_out;          // [NMAX]
    int* nnb_out;
    float* dedr_out;       // [NMAX][3]
    cplx<float>* utot_out; // [NFULL] or nullptr
    unsigned char* pos_row;  // row i of the member's reverse-slot table (pos[i][j] = slot of j in N(i)), or nullptr
};


// All threads of the CTA call it with the same arguments.  at(slot) returns the SBAtom of the
// batch's atom slot (slot < na).  Ends with a CTA barrier.
template <int TJ, class AtomOf, class Side = SBNoSide>
__device__ void sb_batch(const SBShared<TJ>& sh, const SBTables& tb, const SnapDevParams& sp, int na, const AtomOf& at, int n, const double box[3], int* status,
                         bool want_forces, const Side& side = Side(), const SBShape& shape = SBShape()) {
    constexpr int NH = Dims<TJ>::NHALF, NF = Dims<TJ>::NFULL;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float kappa = float(sp.rfac0 * PI / sp.rcut);
    const float rcut = float(sp.rcut);

    const int nwarps = blockDim.x >> 5;   // SB_WARPS or fewer (the CTA size is a tuning knob)
    // U phase
    for (int slot = warp; slot < SB_ATOMS; slot += nwarps) {
        if (slot >= na) {   // empty slot: a zero column keeps the Y phase finite
            for (int f = lane; f < NF; f += 32) sh.ut[f * SB_LD + slot] = make_float2(0.f, 0.f);
            continue;
        }
        const SBAtom A = at(slot);
        int* nb = sh.nbr + slot * NMAX;
        Vec4<float>* dp = sh.disp + slot * NMAX;
        const int cnt = warp_neighbors<float>(nb, dp, lane, n, A.i, A.q64, A.qf, box, sp.rcut, status);
        for (int s = lane; s < cnt; s += 32) {
            A.nbr_out[s] = nb[s];
            if (A.pos_row) A.pos_row[nb[s]] = (unsigned char)s;
        }
        if (lane == 0) {
            *A.nnb_out = cnt;
            sh.nnb[slot] = cnt;
        }
        const int nround = (cnt + 31) / 32;
        float2* lv = sh.lv(warp);
        for (int r = 0; r < (nround > 0 ? nround : 1); ++r)
            sb_u_round<TJ>(lv, sh.ut, dp, sh.tab, lane, slot, r * 32 + lane, cnt, kappa, rcut, sp.switchflag, r == 0);
        for (int e = lane; e < NH; e += 32) {
            const ElemRT<float>& t = sh.tab[e];
            if (t.mir >= 0) {
                const float2 v = sh.ut[t.full * SB_LD + slot];
                const float sg = t.mirneg ? -1.f : 1.f;
                sh.ut[t.mir * SB_LD + slot] = make_float2(sg * v.x, -sg * v.y);
            }
        }
        __syncwarp();
        if (A.utot_out) {
            for (int f = lane; f < NF; f += 32) {
                const float2 v = sh.ut[f * SB_LD + slot];
                A.utot_out[f] = cplx<float>{v.x, v.y};
            }
        }
    }
    __syncthreads();
    if (!want_forces) return;

    sb_y_phase<TJ>(sh, tb, lane, na, side, shape);
    sb_fill_middle<TJ>(sh.yt);

    // dE/dr phase
    for (int slot = warp; slot < na; slot += nwarps) {
        const SBAtom A = at(slot);
        float2* yw = sh.yw(warp);
        sb_weight_y<TJ>(sh.yt, slot, yw, sh.tab, lane);
        __syncwarp();
        const int cnt = sh.nnb[slot];
        const Vec4<float>* dp = sh.disp + slot * NMAX;
        for (int r = 0; r * 32 < cnt; ++r)
            sb_f_round<TJ>(yw, dp, r * 32 + lane, cnt, kappa, rcut, sp.switchflag, A.dedr_out);
        __syncwarp();
    }
    __syncthreads();
}

}  // namespace pmd
