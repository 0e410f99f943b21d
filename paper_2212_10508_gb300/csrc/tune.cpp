// Run-time shape of the batched FP32 fine kernel and its autotuner: a coordinate search over
// the shape knobs (multi-row warp thresholds of the Y contraction, atoms per warp in the
// integrator phase, the Y stage that draws the Gaussian increments, and the CTA size, which
// selects one of two compiled instantiations of the kernel: 16 warps with at most 128 registers
// per thread or 8 warps with up to 255), each candidate timed with CUDA events on a length-scaled
// copy of the caller's batch.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pmd_internal.h"

namespace pmd {
int fine_propagate(pmd_engine* e, int nbatch, int n, double* q, double* v, long stride, const int32_t* nsteps,
                   const int64_t* ids, const pmd_langevin& lp, cudaStream_t st);
int check_langevin_params(const pmd_langevin* lp);
}  // namespace pmd

using namespace pmd;

static int check_tuning(const pmd_fine_tuning* t) {
    if (!t) return fail(PMD_EINVAL, "tuning: NULL");
    if (t->rows2_atoms < 0 || t->rows2_atoms > 16 || t->rows4_atoms < 0 || t->rows4_atoms > 8 || t->b_group < 1 ||
        t->b_group > 10 || t->noise_stage < -1 || t->noise_stage > 15 || (t->warps != 8 && t->warps != 16))
        return fail(PMD_EINVAL, "tuning: rows2_atoms 0..16, rows4_atoms 0..8, b_group 1..10, noise_stage -1..15, "
                                "warps 8 or 16");
    return PMD_OK;
}

extern "C" int pmd_engine_get_tuning(const pmd_engine* e, pmd_fine_tuning* out) {
    if (!e || !out) return fail(PMD_EINVAL, "pmd_engine_get_tuning: NULL argument");
    *out = e->tune;
    return PMD_OK;
}

extern "C" int pmd_engine_set_tuning(pmd_engine* e, const pmd_fine_tuning* t) {
    if (!e) return fail(PMD_EINVAL, "pmd_engine_set_tuning: NULL engine");
    int rc = check_tuning(t);
    if (rc) return rc;
    e->tune = *t;
    return PMD_OK;
}

namespace {
struct TuneBufs {
    DevBuf q0, v0, q, v, L;
    ~TuneBufs() {
        q0.release();
        v0.release();
        q.release();
        v.release();
        L.release();
    }
};
}  // namespace

extern "C" int pmd_engine_autotune(pmd_engine* e, int nbatch, int natoms, const double* q, const double* v,
                                   int64_t member_stride, const int32_t* nsteps, const int64_t* interval_id,
                                   const pmd_langevin* lp, int max_steps, pmd_stream_t stream, pmd_fine_tuning* chosen,
                                   double* best_ms) {
    if (!e) return fail(PMD_EINVAL, "pmd_engine_autotune: NULL engine");
    int rc = check_langevin_params(lp);
    if (rc) return rc;
    if (e->p.fine.precision == PMD_FP64) return fail(PMD_EUNSUPPORTED, "pmd_engine_autotune: the FP64 fine kernel has no shape knobs");
    if (natoms != e->p.natoms || nbatch < 1 || member_stride < 3L * natoms || max_steps < 1)
        return fail(PMD_EINVAL, "pmd_engine_autotune: need natoms == engine natoms, nbatch >= 1, "
                                "member_stride >= 3*natoms, max_steps >= 1");
    if (!q || !v || !nsteps || !interval_id) return fail(PMD_EINVAL, "pmd_engine_autotune: NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = pmd_engine_reserve(e, nbatch))) return rc;

    // interval lengths scaled so that the longest takes max_steps (zero lengths stay zero)
    std::vector<int32_t> L(nbatch);
    PMD_CUDA_TRY(cudaMemcpyAsync(L.data(), nsteps, nbatch * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PMD_CUDA_TRY(cudaStreamSynchronize(st));
    int Lmax = 0;
    for (int x : L) Lmax = std::max(Lmax, x);
    if (Lmax <= 0) return fail(PMD_EINVAL, "pmd_engine_autotune: every interval has zero steps");
    for (int& x : L) x = x <= 0 ? 0 : std::max(1, (int)std::lround((double)x * max_steps / Lmax));

    const size_t row = (size_t)3 * natoms * sizeof(double);
    TuneBufs b;
    if ((rc = b.q0.ensure(nbatch * row)) || (rc = b.v0.ensure(nbatch * row)) || (rc = b.q.ensure(nbatch * row)) ||
        (rc = b.v.ensure(nbatch * row)) || (rc = b.L.ensure(nbatch * sizeof(int32_t))))
        return rc;
    const size_t pitch = (size_t)member_stride * sizeof(double);
    PMD_CUDA_TRY(cudaMemcpy2DAsync(b.q0.p, row, q, pitch, row, nbatch, cudaMemcpyDeviceToDevice, st));
    PMD_CUDA_TRY(cudaMemcpy2DAsync(b.v0.p, row, v, pitch, row, nbatch, cudaMemcpyDeviceToDevice, st));
    PMD_CUDA_TRY(cudaMemcpyAsync(b.L.p, L.data(), nbatch * sizeof(int32_t), cudaMemcpyHostToDevice, st));

    cudaEvent_t t0, t1;
    PMD_CUDA_TRY(cudaEventCreate(&t0));
    PMD_CUDA_TRY(cudaEventCreate(&t1));
    const int saved_profile = e->profile;
    e->profile = 0;
    // one timed run of a shape: best of two after a warm-up launch
    auto time_shape = [&](const pmd_fine_tuning& sh, double* ms) -> int {
        e->tune = sh;
        double best = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            PMD_CUDA_TRY(cudaMemcpyAsync(b.q.p, b.q0.p, nbatch * row, cudaMemcpyDeviceToDevice, st));
            PMD_CUDA_TRY(cudaMemcpyAsync(b.v.p, b.v0.p, nbatch * row, cudaMemcpyDeviceToDevice, st));
            PMD_CUDA_TRY(cudaEventRecord(t0, st));
            int r = fine_propagate(e, nbatch, natoms, b.q.as<double>(), b.v.as<double>(), 3L * natoms,
                                   b.L.as<int32_t>(), interval_id, *lp, st);
            if (r) return r;
            PMD_CUDA_TRY(cudaEventRecord(t1, st));
            PMD_CUDA_TRY(cudaEventSynchronize(t1));
            float f = 0.f;
            PMD_CUDA_TRY(cudaEventElapsedTime(&f, t0, t1));
            if (rep > 0) best = std::min(best, (double)f);
        }
        *ms = best;
        return PMD_OK;
    };
    pmd_fine_tuning best = e->tune;
    double best_t = 0.0;
    rc = time_shape(best, &best_t);
    // coordinate search: each knob in turn over its candidates, keeping the fastest so far
    std::vector<std::vector<int>> cand = {{16, 12, 8, 0}, {8, 4, 0}, {8, 10, 6, 4}, {-1, 2, 4, 5, 1}, {16, 8}};
    if (e->p.fine.twojmax != 8) cand[4] = {16};   // the 8-warp kernel is built for 2J = 8
    for (int knob = 0; knob < 5 && !rc; ++knob)
        for (int val : cand[knob]) {
            pmd_fine_tuning sh = best;
            int* f = knob == 0 ? &sh.rows2_atoms : knob == 1 ? &sh.rows4_atoms : knob == 2 ? &sh.b_group
                                 : knob == 3 ? &sh.noise_stage : &sh.warps;
            if (*f == val) continue;
            *f = val;
            double t = 0.0;
            if ((rc = time_shape(sh, &t))) break;
            if (t < best_t) {
                best_t = t;
                best = sh;
            }
        }
    e->tune = best;
    e->profile = saved_profile;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return pmd_sync_status(e, stream);
}
