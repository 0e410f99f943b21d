// FMA throughput of the device, measured: the denominators of the ALU roofline of the SNAP
// kernels (their Clebsch-Gordan contraction, recursions and force contractions are plain FP32 or
// FP64 FMA arithmetic on data in shared memory and registers).  Every thread runs NCHAIN
// independent FMA chains, so neither latency nor memory bounds the loop; the grid fills every SM
// with 2048 threads.  Results are written only when an impossible value comes out, which keeps
// the chains alive without memory traffic.
#include "pmd_internal.h"

namespace pmd {

static __device__ double g_peak_sink;

constexpr int PEAK_CHAIN = 16;   // independent FMAs per thread and iteration (FP32 lanes)
constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CTAS_PER_SM = 8;

template <int KIND>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(int iters, double a, double b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (KIND == PMD_PEAK_FFMA) {
        const float fa = (float)a, fb = (float)b;
        float x[PEAK_CHAIN];
#pragma unroll
        for (int j = 0; j < PEAK_CHAIN; ++j) x[j] = (float)(t & 7) + 0.125f * j;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < PEAK_CHAIN; ++j) x[j] = fmaf(x[j], fa, fb);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < PEAK_CHAIN; ++j) s += x[j];
        if (s == -1.2345f) g_peak_sink = s;
    } else if constexpr (KIND == PMD_PEAK_FFMA2) {
        const float2 fa = make_float2((float)a, (float)a), fb = make_float2((float)b, (float)b);
        float2 x[PEAK_CHAIN / 2];
#pragma unroll
        for (int j = 0; j < PEAK_CHAIN / 2; ++j) x[j] = make_float2((float)(t & 7) + 0.125f * j, 0.5f * j);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < PEAK_CHAIN / 2; ++j) x[j] = __ffma2_rn(x[j], fa, fb);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < PEAK_CHAIN / 2; ++j) s += x[j].x + x[j].y;
        if (s == -1.2345f) g_peak_sink = s;
    } else {
        double x[PEAK_CHAIN / 2];
#pragma unroll
        for (int j = 0; j < PEAK_CHAIN / 2; ++j) x[j] = (double)(t & 7) + 0.125 * j;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < PEAK_CHAIN / 2; ++j) x[j] = fma(x[j], a, b);
        }
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < PEAK_CHAIN / 2; ++j) s += x[j];
        if (s == -1.2345) g_peak_sink = s;
    }
}

template <int KIND>
static int time_peak(int iters, cudaStream_t st, float* ms, long* fmas) {
    int dev = 0, nsm = 0;
    PMD_CUDA_TRY(cudaGetDevice(&dev));
    PMD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * PEAK_CTAS_PER_SM;
    cudaEvent_t e0, e1;
    PMD_CUDA_TRY(cudaEventCreate(&e0));
    PMD_CUDA_TRY(cudaEventCreate(&e1));
    k_fma_peak<KIND><<<blocks, PEAK_THREADS, 0, st>>>(iters / 8 + 1, 0.999, 1e-3);   // warm-up (clocks, code)
    cudaEventRecord(e0, st);
    k_fma_peak<KIND><<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.999, 1e-3);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "pmd_alu_peak");
    const long per_iter = KIND == PMD_PEAK_DFMA ? PEAK_CHAIN / 2 : PEAK_CHAIN;   // FMAs per thread and iteration
    *fmas = (long)blocks * PEAK_THREADS * per_iter * (long)iters;
    return PMD_OK;
}

}  // namespace pmd

using namespace pmd;

extern "C" int pmd_alu_peak(int kind, double seconds, pmd_stream_t stream, double* tflops, double* ms) {
    if (!tflops || !(seconds > 0) || !(seconds <= 10))
        return fail(PMD_EINVAL, "pmd_alu_peak: need tflops != NULL and 0 < seconds <= 10");
    cudaStream_t st = (cudaStream_t)stream;
    float t = 0.f;
    long fmas = 0;
    // a short probe sizes the timed launch to about `seconds`
    int iters = kind == PMD_PEAK_DFMA ? 256 : 4096;
    for (int round = 0; round < 2; ++round) {
        int rc;
        switch (kind) {
            case PMD_PEAK_FFMA: rc = time_peak<PMD_PEAK_FFMA>(iters, st, &t, &fmas); break;
            case PMD_PEAK_FFMA2: rc = time_peak<PMD_PEAK_FFMA2>(iters, st, &t, &fmas); break;
            case PMD_PEAK_DFMA: rc = time_peak<PMD_PEAK_DFMA>(iters, st, &t, &fmas); break;
            default: return fail(PMD_EINVAL, "pmd_alu_peak: kind must be PMD_PEAK_FFMA, PMD_PEAK_FFMA2 or PMD_PEAK_DFMA");
        }
        if (rc) return rc;
        if (round == 0) {
            const double scale = seconds * 1e3 / (t > 1e-3f ? t : 1e-3f);
            iters = (int)std::min(2.0e9, std::max(1.0, iters * scale));
        }
    }
    *tflops = 2.0 * (double)fmas / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PMD_OK;
}
