// Location of the self-interstitial (Sec. 3: the well of the SIA in each frame, from which the
// residence times in metastable states are counted) by Wigner-Seitz analysis: every atom is
// assigned to the nearest site of a reference lattice shifted by the frame's centre-of-mass
// displacement, and the well is the most occupied site.  The rounding order of every step is
// fixed (see sia_locate in pmd.h) so that each nearest-site decision is reproducible bit for bit.
#include <algorithm>

#include "device_common.cuh"
#include "pmd_internal.h"

namespace pmd {

constexpr int SIA_MAX_SITES = 4096;
constexpr int SIA_THREADS = 256;

// One CTA per frame (grid-stride over frames).  Shared memory: the sites [3][nsites] and the
// occupancy counts [nsites].
__global__ void __launch_bounds__(SIA_THREADS) k_sia_locate(int nf, int n, int ns, double L0, double L1, double L2,
                                                           const double* __restrict__ frames, long stride,
                                                           const double* __restrict__ ref,
                                                           const double* __restrict__ sites, int32_t* __restrict__ well,
                                                           int32_t* __restrict__ occ) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* S = reinterpret_cast<double*>(smem);
    int* cnt = reinterpret_cast<int*>(S + 3 * ns);
    __shared__ double c[3];
    const double L[3] = {L0, L1, L2};
    for (int x = threadIdx.x; x < 3 * ns; x += blockDim.x) S[x] = sites[x];
    for (long f = blockIdx.x; f < nf; f += gridDim.x) {
        const double* q = frames + f * stride;
        for (int s = threadIdx.x; s < ns; s += blockDim.x) cnt[s] = 0;
        if (threadIdx.x < 3) {   // centre-of-mass displacement, summed in index order
            const int a = threadIdx.x;
            double sum = 0.0;
            for (int i = 0; i < n; ++i) sum = __dadd_rn(sum, __dsub_rn(q[a * n + i], ref[a * n + i]));
            c[a] = __ddiv_rn(sum, (double)n);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double p[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) p[a] = __dsub_rn(q[a * n + i], c[a]);
            double best = 0.0;
            int bs = -1;
            for (int s = 0; s < ns; ++s) {
                double d[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    double t = __dsub_rn(p[a], S[a * ns + s]);
                    t = __dsub_rn(t, __dmul_rn(L[a], rint(__ddiv_rn(t, L[a]))));
                    d[a] = t;
                }
                const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
                if (bs < 0 || r2 < best) {   // strict: the smallest index wins a tie
                    best = r2;
                    bs = s;
                }
            }
            atomicAdd(&cnt[bs], 1);
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // most occupied site, smallest index on ties
            int bc = -1, bi = 0;
            for (int s = threadIdx.x; s < ns; s += 32)
                if (cnt[s] > bc) {
                    bc = cnt[s];
                    bi = s;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const int oc = __shfl_xor_sync(0xffffffffu, bc, o), oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oc > bc || (oc == bc && oi < bi)) {
                    bc = oc;
                    bi = oi;
                }
            }
            if (threadIdx.x == 0) {
                well[f] = bi;
                occ[f] = bc;
            }
        }
        __syncthreads();   // cnt and c are rewritten for the next frame
    }
}

}  // namespace pmd

using namespace pmd;

extern "C" int sia_locate(int nframes, int natoms, int nsites, const double box[3], const double* frames,
                          int64_t frame_stride, const double* ref, const double* sites, int32_t* well,
                          int32_t* occupancy, pmd_stream_t stream) {
    if (nframes < 0 || natoms < 1 || nsites < 1 || nsites > SIA_MAX_SITES)
        return fail(PMD_EINVAL, "sia_locate: need nframes >= 0, natoms >= 1 and 1 <= nsites <= 4096");
    if (!box || !(box[0] > 0.0) || !(box[1] > 0.0) || !(box[2] > 0.0))
        return fail(PMD_EINVAL, "sia_locate: box lengths must be positive");
    if (nframes == 0) return PMD_OK;
    if (!frames || !ref || !sites || !well || !occupancy) return fail(PMD_EINVAL, "sia_locate: NULL array");
    if (frame_stride < 3L * natoms) return fail(PMD_EINVAL, "sia_locate: frame_stride < 3 natoms");
    const size_t sm = (size_t)nsites * (3 * sizeof(double) + sizeof(int));
    PMD_CUDA_TRY(cudaFuncSetAttribute(k_sia_locate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0;
    PMD_CUDA_TRY(cudaGetDevice(&dev));
    PMD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(nframes, 4 * nsm);
    k_sia_locate<<<grid, SIA_THREADS, sm, (cudaStream_t)stream>>>(nframes, natoms, nsites, box[0], box[1], box[2],
                                                                 frames, (long)frame_stride, ref, sites, well,
                                                                 occupancy);
    PMD_CUDA_TRY(cudaGetLastError());
    return PMD_OK;
}

extern "C" int sia_residence(const int32_t* well, int nframes, int capacity, int32_t* lengths, int32_t* sites,
                             int* nruns) {
    if (!well || !nruns || nframes < 0 || capacity < 0)
        return fail(PMD_EINVAL, "sia_residence: need well, nruns, nframes >= 0 and capacity >= 0");
    int k = 0, start = 0;
    for (int f = 1; f < nframes; ++f) {
        if (well[f] == well[f - 1]) continue;
        if (k >= capacity) return fail(PMD_ENOMEM, "sia_residence: capacity too small");
        if (lengths) lengths[k] = f - start;
        if (sites) sites[k] = well[f - 1];
        ++k;
        start = f;
    }
    *nruns = k;
    return PMD_OK;
}
