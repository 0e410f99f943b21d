// Kernels of the standalone SNAP energy/force call (snap_energy_forces) and their launch:
// neighbour lists, U_tot, the adjoint and the pair derivatives per atom (k_snap_atoms), the force
// gather, the bispectrum and the energy sums.  Included by snap.cu (band limits 2J <= 8) and by
// snap_large.cu (2J = 10, 12, 14, FP64), so that the two sets compile in parallel; every kernel
// has internal linkage in each translation unit.
#pragma once

#include <algorithm>

#include "eam_device.cuh"   // wrap_f32
#include "pmd_internal.h"
#include "snap_kernels.cuh"

namespace pmd {

SnapView snap_view(const pmd_snap* s, const double* beta);


static __global__ void k_wrap_f32(const double* __restrict__ pos, int nbatch, int n, double b0, double b1, double b2,
                           float4* __restrict__ qf) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nbatch * n) return;
    const long bb = idx / n, i = idx % n;
    const double* P = pos + bb * 3 * n;
    double x = P[i], y = P[n + i], z = P[2 * n + i];
    const double box[3] = {b0, b1, b2};
    qf[idx] = wrap_f32(x, y, z, box);
}

template <typename real, int TJ>
static __global__ void __launch_bounds__(snap_cta_threads<real, TJ>(), 1)
    k_snap_atoms(SnapView v, int nbatch, int n, double b0, double b1, double b2, const double* __restrict__ pos,
                 const float4* __restrict__ qf, int* __restrict__ nbr, int* __restrict__ nnb, real* __restrict__ dedr,
                 cplx<real>* __restrict__ utot, int* status, int want_forces) {
    extern __shared__ __align__(16) unsigned char smem[];
    const double box[3] = {b0, b1, b2};
    const long natoms_all = (long)nbatch * n;
    if constexpr (sizeof(real) == 4) {
        // batched design: CTA c evaluates the contiguous range of atoms [c0, c1) in batches of 32
        SBShared<TJ> sh = sb_shared_carve<TJ>(smem, v);
        sb_shared_load<TJ>(sh, v);
        __syncthreads();
        const long chunk = (natoms_all + gridDim.x - 1) / gridDim.x;
        const long c0 = (long)blockIdx.x * chunk;
        const long c1 = c0 + chunk < natoms_all ? c0 + chunk : natoms_all;
        for (long bs = c0; bs < c1; bs += SB_ATOMS) {
            const int na = (int)(c1 - bs < SB_ATOMS ? c1 - bs : SB_ATOMS);
            auto at = [&](int slot) {
                const long item = bs + slot;
                const long bb = item / n;
                return SBAtom{pos + bb * 3 * n, qf + bb * n, (int)(item % n), nbr + item * NMAX, nnb + item,
                              dedr + item * NMAX * 3, utot ? utot + item * Dims<TJ>::NFULL : nullptr, nullptr};
            };
            sb_batch<TJ>(sh, sb_tables(v), v.sp, na, at, n, box, status, want_forces != 0);
        }
    } else {
        SnapShared<real, TJ> sh = snap_shared_carve<real, TJ>(smem, v);
        snap_shared_load<real, TJ>(sh, v);
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
        for (long item = (long)blockIdx.x * (blockDim.x >> 5) + warp; item < natoms_all; item += nwarps) {
            const long bb = item / n;
            const int i = (int)(item % n);
            snap_atom_warp2<real, TJ>(sh.ws[warp], sh.tab, v.yt, sh.cg, sh.beff, v.sp, lane, n, i, pos + bb * 3 * n,
                                      qf + bb * n, box, nbr + item * NMAX, nnb + item, dedr + item * NMAX * 3,
                                      utot ? utot + item * Dims<TJ>::NFULL : nullptr, status, want_forces != 0);
        }
    }
}

// B_t of one atom from U_tot (full layout): Re sum_{m m'} conj(U^j) Z^j_{j1 j2}, FP64 accumulation.
// Thread (t, atom), triple-major: the 32 lanes of a warp take 32 atoms of the same triple, so every
// loop bound and Clebsch-Gordan index is warp-uniform.  FP64 mode: every operation in FP64.
// FP32-bulk mode: each element Z(m, m') (a Clebsch-Gordan double sum of at most (j1+1)^2 products)
// in FP32, and the sum of conj(U) Z over the elements in double-float arithmetic (FP64-class
// accuracy on the FP32 pipes; an FP64 instruction costs as much as dozens of FP32 ones on this
// part), converted to FP64 once per component.
template <typename real, int TJ>
static __global__ void k_snap_bispectrum(const cplx<real>* __restrict__ utot, long natoms_all, int nB,
                                  const int4* __restrict__ triblk, const real* __restrict__ cg,
                                  const int4* __restrict__ blk, double* __restrict__ Bout) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= natoms_all * nB) return;
    const int t = (int)(idx / natoms_all);
    const long ia = idx - (long)t * natoms_all;
    const int4 tb = triblk[t];
    const int ta = tb.y, tbb = tb.z, tj = tb.w;
    const int4 bk = blk[tb.x];
    const real* c = cg + bk.w;
    const cplx<real>* U = utot + ia * Dims<TJ>::NFULL;
    const cplx<real>* Ua = U + f_off(ta);
    const cplx<real>* Ub = U + f_off(tbb);
    const cplx<real>* Uj = U + f_off(tj);
    const int s = (ta + tbb - tj) / 2;
    double B = 0.0;
    if constexpr (sizeof(real) == 4) {
        FF Bf{0.f, 0.f};
        for (int p = 0; p <= tj; ++p)
            for (int q = 0; q <= tj; ++q) {
                float zr = 0.f, zi = 0.f;
                for (int p1 = max(0, p + s - tbb); p1 <= min(ta, p + s); ++p1) {
                    const int p2 = p + s - p1;
                    const float c1 = c[p1 * (tbb + 1) + p2];
                    for (int q1 = max(0, q + s - tbb); q1 <= min(ta, q + s); ++q1) {
                        const int q2 = q + s - q1;
                        const float cc = c1 * c[q1 * (tbb + 1) + q2];
                        const cplx<real> x = Ua[p1 * (ta + 1) + q1], y = Ub[p2 * (tbb + 1) + q2];
                        zr = fmaf(cc, x.re * y.re - x.im * y.im, zr);
                        zi = fmaf(cc, x.re * y.im + x.im * y.re, zi);
                    }
                }
                const cplx<real> u = Uj[p * (tj + 1) + q];
                Bf = ff_add(Bf, ff_two_sum(u.re * zr, u.im * zi));
            }
        B = (double)Bf.hi + (double)Bf.lo;
    } else {
        for (int p = 0; p <= tj; ++p)
            for (int q = 0; q <= tj; ++q) {
                double zr = 0, zi = 0;
                for (int p1 = max(0, p + s - tbb); p1 <= min(ta, p + s); ++p1) {
                    const int p2 = p + s - p1;
                    const double c1 = (double)c[p1 * (tbb + 1) + p2];
                    for (int q1 = max(0, q + s - tbb); q1 <= min(ta, q + s); ++q1) {
                        const int q2 = q + s - q1;
                        const double cc = c1 * (double)c[q1 * (tbb + 1) + q2];
                        const cplx<real> x = Ua[p1 * (ta + 1) + q1], y = Ub[p2 * (tbb + 1) + q2];
                        const double xr = x.re, xi = x.im, yr = y.re, yi = y.im;
                        zr += cc * (xr * yr - xi * yi);
                        zi += cc * (xr * yi + xi * yr);
                    }
                }
                const cplx<real> u = Uj[p * (tj + 1) + q];
                B += (double)u.re * zr + (double)u.im * zi;
            }
    }
    Bout[ia * nB + t] = B;
}

template <typename real>
static __global__ void k_snap_gather(const int* __restrict__ nbr, const int* __restrict__ nnb,
                              const real* __restrict__ dedr, int nbatch, int n, double* __restrict__ forces,
                              int* status) {
    // one warp per atom
    const long idx = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (idx >= (long)nbatch * n) return;
    const long bb = idx / n;
    const int k = (int)(idx % n);
    double F[3];
    warp_gather_force<real>(nbr + bb * n * NMAX, nnb + bb * n, dedr + bb * n * NMAX * 3, k, lane, F, status);
    if (lane < 3) forces[bb * 3 * n + (long)lane * n + k] = F[lane == 0 ? 0 : (lane == 1 ? 1 : 2)];
}

// per member: E = sum_i (beta_0 + sum_t beta_t B_it), sumB[t] = sum_i B_it.  One CTA of
// SNAP_E_THREADS per member: thread t sums column t of B over the atoms (sumB); for E every thread
// sums the E_i of atoms i = thread, thread + SNAP_E_THREADS, ... and the partial sums are combined
// by a fixed binary tree in shared memory.  Every sum runs in a fixed order: deterministic.
constexpr int SNAP_E_THREADS = 128;

static __global__ void __launch_bounds__(SNAP_E_THREADS) k_snap_energy(const double* __restrict__ B, int nbatch, int n,
                                                                 int nB, const double* __restrict__ beta,
                                                                 double* __restrict__ energy,
                                                                 double* __restrict__ sumB) {
    __shared__ double part[SNAP_E_THREADS];
    const int bb = blockIdx.x;
    const double* Bm = B + (long)bb * n * nB;
    if (sumB) {
        for (int t = threadIdx.x; t < nB; t += blockDim.x) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += Bm[(long)i * nB + t];
            sumB[(long)bb * (1 + nB) + 1 + t] = s;
        }
        if (threadIdx.x == 0) sumB[(long)bb * (1 + nB)] = (double)n;
    }
    if (!energy) return;
    double e = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double Ei = beta[0];
        for (int t = 0; t < nB; ++t) Ei += beta[1 + t] * Bm[(long)i * nB + t];
        e += Ei;
    }
    part[threadIdx.x] = e;
    __syncthreads();
    for (int w = SNAP_E_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) energy[bb] = part[0];
}

template <typename real, int TJ>
static int launch_snap(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                       double* energy, double* forces, double* sumB, const SnapScratch& sc, cudaStream_t st) {
    const long na = (long)nbatch * n;
    SnapView v = snap_view(s, beta);
    const bool want_B = energy || sumB;
    float4* qf = sc.qf;
    if (sizeof(real) == 4) {
        k_wrap_f32<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(pos, nbatch, n, box[0], box[1], box[2], qf);
        PMD_CUDA_TRY(cudaGetLastError());
    }
    const bool batched = sizeof(real) == 4;
    const size_t sm = batched ? sb_shared_bytes<TJ>(v) : snap_shared_bytes<real, TJ>(v);
    constexpr int threads = snap_cta_threads<real, TJ>();
    PMD_CUDA_TRY(cudaFuncSetAttribute(k_snap_atoms<real, TJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    long blocks;
    if (batched) {
        int dev = 0, nsm = 0;
        PMD_CUDA_TRY(cudaGetDevice(&dev));
        PMD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        blocks = std::min<long>((na + SB_ATOMS - 1) / SB_ATOMS, std::max(1, nsm));
    } else {
        blocks = (na + threads / 32 - 1) / (threads / 32);
    }
    k_snap_atoms<real, TJ><<<(unsigned)blocks, threads, sm, st>>>(
        v, nbatch, n, box[0], box[1], box[2], pos, qf, sc.nbr, sc.nnb, static_cast<real*>(sc.dedr),
        want_B ? static_cast<cplx<real>*>(sc.utot) : nullptr, s->s_status.as<int>(), forces != nullptr);
    PMD_CUDA_TRY(cudaGetLastError());
    if (forces) {
        k_snap_gather<real><<<(unsigned)((na + 7) / 8), 256, 0, st>>>(
            sc.nbr, sc.nnb, static_cast<const real*>(sc.dedr), nbatch, n, forces, s->s_status.as<int>());
        PMD_CUDA_TRY(cudaGetLastError());
    }
    if (want_B) {
        const long nt = na * s->T.nB;
        k_snap_bispectrum<real, TJ><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(
            static_cast<const cplx<real>*>(sc.utot), na, s->T.nB, s->d_triblk.as<int4>(), s->d_cg.as<real>(),
            s->d_blk.as<int4>(), sc.B);
        PMD_CUDA_TRY(cudaGetLastError());
        k_snap_energy<<<nbatch, SNAP_E_THREADS, 0, st>>>(sc.B, nbatch, n, s->T.nB, beta, energy, sumB);
        PMD_CUDA_TRY(cudaGetLastError());
    }
    return PMD_OK;
}

}  // namespace pmd
