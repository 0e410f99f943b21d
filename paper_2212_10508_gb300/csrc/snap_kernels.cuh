// Shared-memory layout of the SNAP kernels: per-CTA tables (Clebsch-Gordan blocks, beta_eff)
// followed by one WarpScratch2 per warp.
#pragma once

#include "snap_v2.cuh"

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
    const double* beta;
    int ncg, nblk, nB;
    SnapDevParams sp;
};

template <typename real, int TJ>
struct SnapShared {
    real* cg;
    real* beff;
    WarpScratch2<real, TJ>* ws;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename real, int TJ>
__host__ __device__ inline size_t snap_table_bytes(const SnapView& v) {
    size_t o = 0;
    o = align_up(o + (size_t)v.ncg * sizeof(real), 32);
    o = align_up(o + (size_t)v.nblk * sizeof(real), 32);
    return o;
}

template <typename real, int TJ>
__host__ __device__ inline size_t snap_shared_bytes(const SnapView& v, int nwarps = SNAP_THREADS / 32) {
    return snap_table_bytes<real, TJ>(v) + (size_t)nwarps * sizeof(WarpScratch2<real, TJ>);
}

template <typename real, int TJ>
__device__ inline SnapShared<real, TJ> snap_shared_carve(unsigned char* smem, const SnapView& v) {
    SnapShared<real, TJ> sh;
    size_t o = 0;
    sh.cg = reinterpret_cast<real*>(smem + o);
    o = align_up(o + (size_t)v.ncg * sizeof(real), 32);
    sh.beff = reinterpret_cast<real*>(smem + o);
    o = align_up(o + (size_t)v.nblk * sizeof(real), 32);
    sh.ws = reinterpret_cast<WarpScratch2<real, TJ>*>(smem + o);
    return sh;
}

// Copy the CG tables into shared memory and form beta_eff(block) = sum coef * beta[1+t]
// (per block a short fixed-order sum: deterministic).
template <typename real, int TJ>
__device__ inline void snap_shared_load(SnapShared<real, TJ>& sh, const SnapView& v) {
    const real* cg = reinterpret_cast<const real*>(v.cg);
    for (int x = threadIdx.x; x < v.ncg; x += blockDim.x) sh.cg[x] = cg[x];
    for (int b = threadIdx.x; b < v.nblk; b += blockDim.x) {
        double s = 0.0;
        for (int c = v.beffptr[b]; c < v.beffptr[b + 1]; ++c) s += v.beffc[c] * v.beta[1 + v.befft[c]];
        sh.beff[b] = (real)s;
    }
}

}  // namespace pmd
