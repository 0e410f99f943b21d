// Test helper: draws raw Philox4x32-10 blocks with cuRAND's device API (curand_kernel.h), so that
// the oracle's Philox can be compared, word for word, with an implementation it shares nothing
// with.  cuRAND's state for (seed, subsequence, offset = 4 t) produces as its first curand4()
// the block of counter (t_lo, t_hi, subsequence_lo, subsequence_hi) under key (seed_lo, seed_hi).
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>

static __global__ void k_curand_philox(int n, const unsigned long long* seed, const unsigned long long* subseq,
                                       const unsigned long long* block, uint32_t* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], subseq[i], 4ull * block[i], &st);
    uint4 r = curand4(&st);
    out[4 * i + 0] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

// All pointers are device pointers of n elements (out: 4 n words).  Returns a cudaError_t.
extern "C" int curand_philox_blocks(int n, const unsigned long long* seed, const unsigned long long* subseq,
                                    const unsigned long long* block, uint32_t* out) {
    if (n <= 0) return 0;
    k_curand_philox<<<(n + 127) / 128, 128>>>(n, seed, subseq, block, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return (int)e;
}
