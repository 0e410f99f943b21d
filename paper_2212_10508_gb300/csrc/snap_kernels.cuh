// Shared-memory layout of the SNAP kernels: per-CTA tables (Clebsch-Gordan blocks, beta_eff)
// followed by one WarpScratch2 per warp.
#pragma once

#include "snap_batch.cuh"

namespace pmd {

#ifndef SNAP_THREADS
#define SNAP_THREADS 256
#endif

struct SnapView {
    const void* cg;
    const int* beffptr;
    const int* befft;
    const double* beffc;
    SnapV2Tables yt;
    const int4* sbjobs;      // batched Y phase jobs (FP32 design)
    const int2* sbrows;      // job range of each (stage, row)
    const int* sbsptr;       // row ranges of the stages
    const float* sbcoef;     // per-job Clebsch-Gordan weights
    const int2* sbgroups;    // row groups (first row, count) for multi-row warps
    const int* sbgptr;       // [2][nstages][2] group ranges per stage (R = 2, 4)
    const double* beta;
    int ncg, nblk, nB;
    SnapDevParams sp;
};

template <typename real, int TJ>
struct SnapShared {
    real* cg;
    real* beff;
    ElemRT<real>* tab;
    WarpScratch2<real, TJ>* ws;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The Clebsch-Gordan values sit in shared memory up to 2J = 8; from 2J = 10 on (80 KB and more)
// the kernels read them from global memory through the caches.
template <int TJ>
__host__ __device__ constexpr bool snap_cg_shared() { return TJ <= 8; }

template <typename real, int TJ>
__host__ __device__ inline size_t snap_table_bytes(const SnapView& v) {
    size_t o = 0;
    if (snap_cg_shared<TJ>()) o = align_up(o + (size_t)v.ncg * sizeof(real), 32);
    o = align_up(o + (size_t)v.nblk * sizeof(real), 32);
    o = align_up(o + (size_t)Dims<TJ>::NHALF * sizeof(ElemRT<real>), 32);
    return o;
}

// threads per CTA of the SNAP kernels: the batched FP32 design, or one warp per atom (FP64; two
// warps per CTA from 2J = 10 on, whose per-warp scratch is 27-62 KB)
template <typename real, int TJ = 8>
__host__ __device__ constexpr int snap_cta_threads() {
    return sizeof(real) == 4 ? SB_THREADS : (TJ <= 8 ? SNAP_THREADS : 64);
}

template <typename real, int TJ>
__host__ __device__ inline size_t snap_shared_bytes(const SnapView& v, int nwarps = snap_cta_threads<real, TJ>() / 32) {
    return snap_table_bytes<real, TJ>(v) + (size_t)nwarps * sizeof(WarpScratch2<real, TJ>);
}

template <typename real, int TJ>
__device__ inline SnapShared<real, TJ> snap_shared_carve(unsigned char* smem, const SnapView& v) {
    SnapShared<real, TJ> sh;
    size_t o = 0;
    if (snap_cg_shared<TJ>()) {
        sh.cg = reinterpret_cast<real*>(smem + o);
        o = align_up(o + (size_t)v.ncg * sizeof(real), 32);
    } else {
        sh.cg = const_cast<real*>(reinterpret_cast<const real*>(v.cg));
    }
    sh.beff = reinterpret_cast<real*>(smem + o);
    o = align_up(o + (size_t)v.nblk * sizeof(real), 32);
    sh.tab = reinterpret_cast<ElemRT<real>*>(smem + o);
    o = align_up(o + (size_t)Dims<TJ>::NHALF * sizeof(ElemRT<real>), 32);
    sh.ws = reinterpret_cast<WarpScratch2<real, TJ>*>(smem + o);
    return sh;
}

// Copy the CG tables into shared memory and form beta_eff(block) = sum coef * beta[1+t]
// (per block a short fixed-order sum: deterministic).
template <typename real, int TJ>
__device__ inline void snap_shared_load(SnapShared<real, TJ>& sh, const SnapView& v) {
    const real* cg = reinterpret_cast<const real*>(v.cg);
    if (snap_cg_shared<TJ>())
        for (int x = threadIdx.x; x < v.ncg; x += blockDim.x) sh.cg[x] = cg[x];
    for (int b = threadIdx.x; b < v.nblk; b += blockDim.x) {
        double s = 0.0;
        for (int c = v.beffptr[b]; c < v.beffptr[b + 1]; ++c) s += v.beffc[c] * v.beta[1 + v.befft[c]];
        sh.beff[b] = (real)s;
    }
    fill_elem_table<real, TJ>(sh.tab);
}

// ---- batched FP32 design (snap_batch.cuh) ----------------------------------------------------
template <int TJ>
__host__ __device__ inline size_t sb_shared_bytes(const SnapView& v) {
    size_t o = 0;
    o = align_up(o + (size_t)v.nblk * sizeof(float), 32);
    o = align_up(o + (size_t)Dims<TJ>::NHALF * sizeof(ElemRT<float>), 32);
    o = align_up(o + sb_ut_elems<TJ>() * sizeof(float2), 32);
    o = align_up(o + sb_yt_elems<TJ>() * sizeof(float2), 32);
    o = align_up(o + (size_t)SB_ATOMS * NMAX * sizeof(int), 32);
    o = align_up(o + (size_t)SB_ATOMS * sizeof(int), 32);
    o = align_up(o + (size_t)SB_MAX_STAGES * sizeof(int), 32);
    o = align_up(o + (size_t)SB_ATOMS * NMAX * sizeof(Vec4<float>), 32);
    return o;
}

template <int TJ>
__device__ inline SBShared<TJ> sb_shared_carve(unsigned char* smem, const SnapView& v) {
    SBShared<TJ> sh;
    size_t o = 0;
    sh.beff = reinterpret_cast<float*>(smem + o);
    o = align_up(o + (size_t)v.nblk * sizeof(float), 32);
    sh.tab = reinterpret_cast<ElemRT<float>*>(smem + o);
    o = align_up(o + (size_t)Dims<TJ>::NHALF * sizeof(ElemRT<float>), 32);
    sh.ut = reinterpret_cast<float2*>(smem + o) + SB_GUARD * SB_LD;
    o = align_up(o + sb_ut_elems<TJ>() * sizeof(float2), 32);
    sh.yt = reinterpret_cast<float2*>(smem + o);
    o = align_up(o + sb_yt_elems<TJ>() * sizeof(float2), 32);
    sh.nbr = reinterpret_cast<int*>(smem + o);
    o = align_up(o + (size_t)SB_ATOMS * NMAX * sizeof(int), 32);
    sh.nnb = reinterpret_cast<int*>(smem + o);
    o = align_up(o + (size_t)SB_ATOMS * sizeof(int), 32);
    sh.ctr = reinterpret_cast<int*>(smem + o);
    o = align_up(o + (size_t)SB_MAX_STAGES * sizeof(int), 32);
    sh.disp = reinterpret_cast<Vec4<float>*>(smem + o);
    return sh;
}

template <int TJ>
__device__ inline void sb_shared_load(SBShared<TJ>& sh, const SnapView& v) {
    for (int b = threadIdx.x; b < v.nblk; b += blockDim.x) {
        double s = 0.0;
        for (int c = v.beffptr[b]; c < v.beffptr[b + 1]; ++c) s += v.beffc[c] * v.beta[1 + v.befft[c]];
        sh.beff[b] = (float)s;
    }
    fill_elem_table<float, TJ>(sh.tab);
    for (int x = threadIdx.x; x < SB_GUARD * SB_LD; x += blockDim.x) {
        sh.ut[x - SB_GUARD * SB_LD] = make_float2(0.f, 0.f);
        sh.ut[(size_t)Dims<TJ>::NFULL * SB_LD + x] = make_float2(0.f, 0.f);
    }
}

inline __host__ __device__ SBTables sb_tables(const SnapView& v) {
    return SBTables{v.sbjobs, v.sbrows, v.sbsptr, v.sbcoef, v.sbgroups, v.sbgptr};
}

}  // namespace pmd
