// eam_energy_forces: Finnis-Sinclair energies and forces (coarse potential, Sec. 3.1), one CTA
// per system, everything in shared memory (no scratch).
#include <algorithm>

#include "eam_device.cuh"
#include "pmd_internal.h"

namespace pmd {

FSDev make_fs(const pmd_fs_params& p);

template <typename real>
__global__ void __launch_bounds__(512) k_eam_standalone(int n, double b0, double b1, double b2, FSDev fs, const double* __restrict__ pos,
                                 double* __restrict__ energy, double* __restrict__ forces) {
    extern __shared__ __align__(16) unsigned char smem[];
    EamShared s;
    s.q = reinterpret_cast<double*>(smem);
    s.F = s.q + 3 * n;
    s.dF = s.F + 3 * n;
    double* Eat = s.dF + n;
    s.qf = reinterpret_cast<float4*>((reinterpret_cast<size_t>(Eat + n) + 15) / 16 * 16);
    s.nbl = nullptr;   // one evaluation: scan all atoms
    s.nbc = nullptr;
    s.qref = nullptr;
    s.pg = nullptr;
    s.pj = nullptr;
    s.pgc = nullptr;
    const double box[3] = {b0, b1, b2};
    const long m = blockIdx.x;
    const double* P = pos + m * 3 * n;
    for (int x = threadIdx.x; x < 3 * n; x += blockDim.x) s.q[x] = P[x];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.qf[i] = wrap_f32(s.q[i], s.q[n + i], s.q[2 * n + i], box);
    __syncthreads();
    eam_forces_cta<real>(s, n, box, fs, Eat);
    if (forces) {
        double* F = forces + m * 3 * n;
        for (int x = threadIdx.x; x < 3 * n; x += blockDim.x) F[x] = s.F[x];
    }
    if (energy && threadIdx.x == 0) {
        double E = 0.0;
        for (int i = 0; i < n; ++i) E += Eat[i];
        energy[m] = E;
    }
}

int eam_launch(const pmd_fs_params& p, int nbatch, int n, const double box[3], const double* pos, double* energy,
               double* forces, cudaStream_t st) {
    // the launch shape of the coarse propagation kernels: two threads per atom up to 256 atoms
    const int threads = std::min(512, ((2 * n <= 512 ? 2 * n : n) + 31) / 32 * 32);
    const size_t sm = (size_t)n * (3 * 8 + 3 * 8 + 8 + 8 + 16) + 64;
    const FSDev fs = make_fs(p);
    auto go = [&](auto kern) -> int {
        PMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        kern<<<nbatch, threads, sm, st>>>(n, box[0], box[1], box[2], fs, pos, energy, forces);
        PMD_CUDA_TRY(cudaGetLastError());
        return PMD_OK;
    };
    return p.precision == PMD_FP64 ? go(k_eam_standalone<double>) : go(k_eam_standalone<float>);
}

}  // namespace pmd
