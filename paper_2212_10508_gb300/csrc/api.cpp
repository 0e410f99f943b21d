// C ABI entry points: argument validation, contexts, scratch, status reporting.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "pmd_internal.h"

namespace pmd {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t err, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")");
    return err == cudaErrorMemoryAllocation ? PMD_ENOMEM : PMD_ECUDA;
}

int status_to_code(int bits) {
    if (bits & ST_TIMEOUT) return fail(PMD_ETIMEOUT, "a bounded device wait timed out; outputs are invalid");
    if (bits & ST_BADARG) return fail(PMD_EINVAL, "a device-side argument was invalid (negative nsteps, or L1_SYM with nsteps > 1)");
    if (bits & ST_NONFINITE) return fail(PMD_ENONFINITE, "a position or velocity became non-finite");
    if (bits & ST_LOSTATOM) return fail(PMD_ELOSTATOM, "an atom moved more than half a box edge in one step");
    if (bits & ST_NEIGH) return fail(PMD_ENEIGH, "an atom exceeded PMD_MAX_NEIGHBORS neighbours");
    if (bits & ST_BADNEIGH) return fail(PMD_ECUDA, "internal: asymmetric neighbour lists");
    return PMD_OK;
}

int DevBuf::ensure(size_t need) {
    if (need <= bytes) return PMD_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    bytes = need;
    return PMD_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

// implemented in the .cu files
int snap_upload(pmd_snap* s);
int snap_reserve_impl(pmd_snap* s, long na);
int snap_compute(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                 double* energy, double* forces, double* sumB, cudaStream_t st);
int eam_launch(const pmd_fs_params& p, int nbatch, int n, const double box[3], const double* pos, double* energy,
               double* forces, cudaStream_t st);
int fine_propagate(pmd_engine* e, int nbatch, int n, double* q, double* v, long stride, const int32_t* nsteps,
                   const int64_t* ids, const pmd_langevin& lp, cudaStream_t st);
int coarse_propagate(pmd_engine* e, int nbatch, int n, double* q, double* v, long stride, const int32_t* nsteps,
                     const int64_t* ids, const pmd_langevin& lp, cudaStream_t st);
int parareal_sweep(pmd_engine* e, int n_in, int n_fin, const double* jumps, const double* prev, double* cur,
                   double* cout, double delta_expl, int metric, int L, const pmd_langevin& lp, double* delta_host,
                   int* n_stop_host, cudaStream_t st);
int jumps_launch(long count, const double* f, const double* c, double* j, int num_sms, cudaStream_t st);

static int check_snap_params(const pmd_snap_params* p) {
    if (!p) return fail(PMD_EINVAL, "SNAP parameters are NULL");
    if (p->twojmax < 2 || p->twojmax > PMD_MAX_TWOJMAX || (p->twojmax & 1))
        return fail(PMD_EUNSUPPORTED, "twojmax must be 2, 4, ..., 14");
    if (p->twojmax > 8 && p->precision != PMD_FP64)
        return fail(PMD_EUNSUPPORTED, "twojmax > 8 is available in FP64 only");
    if (!(p->rcut > 0) || !(p->rfac0 > 0 && p->rfac0 <= 1) || p->rmin0 != 0.0)
        return fail(PMD_EINVAL, "need rcut > 0, 0 < rfac0 <= 1 and rmin0 == 0");
    if (p->switchflag != 0 && p->switchflag != 1) return fail(PMD_EINVAL, "switchflag must be 0 or 1");
    if (p->precision != PMD_FP64 && p->precision != PMD_FP32_BULK) return fail(PMD_EINVAL, "bad SNAP precision");
    return PMD_OK;
}

static int check_fs(const pmd_fs_params* p) {
    if (!p) return fail(PMD_EINVAL, "EAM parameters are NULL");
    if (!(p->d > 0) || !(p->c > 0) || !std::isfinite(p->A) || !std::isfinite(p->c0) || !std::isfinite(p->c1) ||
        !std::isfinite(p->c2))
        return fail(PMD_EINVAL, "bad Finnis-Sinclair parameters");
    if (p->precision != PMD_FP64 && p->precision != PMD_FP32_BULK) return fail(PMD_EINVAL, "bad EAM precision");
    return PMD_OK;
}

int check_box(const double box[3], double rc) {
    if (!box) return fail(PMD_EINVAL, "box is NULL");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 2.0 * rc) || !std::isfinite(box[a]))
            return fail(PMD_EINVAL, "every box edge must be finite and exceed twice the cutoff");
    return PMD_OK;
}

static int check_langevin(const pmd_langevin* lp) {
    if (!lp) return fail(PMD_EINVAL, "Langevin parameters are NULL");
    if (!(lp->dt > 0) || !(lp->gamma >= 0) || !(lp->T >= 0) || !(lp->mass > 0) || !std::isfinite(lp->dt) ||
        !std::isfinite(lp->gamma) || !std::isfinite(lp->T))
        return fail(PMD_EINVAL, "need dt > 0, gamma >= 0, T >= 0, mass > 0");
    if (lp->scheme != PMD_SCHEME_PAPER && lp->scheme != PMD_SCHEME_BAOAB) return fail(PMD_EINVAL, "bad scheme");
    if (lp->schedule < PMD_SCHED_NONE || lp->schedule > PMD_SCHED_L1_SYM) return fail(PMD_EINVAL, "bad schedule");
    return PMD_OK;
}

int check_langevin_params(const pmd_langevin* lp) { return check_langevin(lp); }

static int read_status(int* dstatus, cudaStream_t st) {
    int h = 0;
    PMD_CUDA_TRY(cudaMemcpyAsync(&h, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
    PMD_CUDA_TRY(cudaStreamSynchronize(st));
    PMD_CUDA_TRY(cudaMemsetAsync(dstatus, 0, sizeof(int), st));
    PMD_CUDA_TRY(cudaStreamSynchronize(st));
    return status_to_code(h);
}

int selftest_waits(pmd_engine* e, long long polls, cudaStream_t st);
int noalloc_scratch_address(void** out);
}  // namespace pmd

using namespace pmd;

extern "C" {

const char* pmd_last_error(void) { return g_last_error.c_str(); }

int pmd_snap_create(const pmd_snap_params* p, pmd_snap** out) {
    if (!out) return fail(PMD_EINVAL, "pmd_snap_create: out is NULL");
    *out = nullptr;
    int rc = check_snap_params(p);
    if (rc) return rc;
    pmd_snap* s = new (std::nothrow) pmd_snap();
    if (!s) return fail(PMD_ENOMEM, "pmd_snap_create: out of host memory");
    s->p = *p;
    cudaGetDevice(&s->device);
    // noalloc_scratch_address also loads the module that holds the static scratch array of
    // snap_energy_forces_noalloc, so that its device memory is reserved here (where allocating
    // is allowed) and not by the first allocation-free call.
    void* noalloc_base = nullptr;
    if ((rc = build_snap_tables(p->twojmax, &s->T)) || (rc = snap_upload(s)) || (rc = s->s_status.ensure(sizeof(int))) ||
        (rc = noalloc_scratch_address(&noalloc_base))) {
        pmd_snap_destroy(s);
        return rc;
    }
    cudaError_t e = cudaMemset(s->s_status.p, 0, sizeof(int));
    if (e != cudaSuccess) {
        pmd_snap_destroy(s);
        return cuda_fail(e, "cudaMemset");
    }
    *out = s;
    return PMD_OK;
}

int pmd_snap_destroy(pmd_snap* s) {
    if (!s) return PMD_OK;
    DevBuf* bufs[] = {&s->d_cg, &s->d_blk, &s->d_beffptr, &s->d_befft, &s->d_beffc, &s->d_jobs,
                      &s->d_roundtb, &s->d_triblk, &s->s_nbr, &s->s_nnb, &s->s_dedr, &s->s_qf, &s->s_utot,
                      &s->s_B, &s->s_status, &s->d_sbjobs, &s->d_sbrows, &s->d_sbsptr, &s->d_sbcoef,
                      &s->d_sbgroups, &s->d_sbgptr};
    for (DevBuf* b : bufs) b->release();
    delete s;
    return PMD_OK;
}

int pmd_snap_num_coeffs(const pmd_snap* s) {
    if (!s) return fail(PMD_EINVAL, "pmd_snap_num_coeffs: NULL context");
    return 1 + s->T.nB;
}

int pmd_snap_flop_model(const pmd_snap* s, double* per_pair, double* per_atom) {
    if (!s) return fail(PMD_EINVAL, "pmd_snap_flop_model: NULL context");
    const double nh = (double)s->T.nhalf;
    // per neighbour, per half element: U pass = recursion (two complex products 12, two scaled
    // adds 4) + weighting 2 + the sum over neighbours 2; dE/dr pass = recursion 16 + contraction
    // with the four weighted Y copies (2 + 2 + 4 + 4); plus ~100 for the final 3-component step
    const double pair = nh * (16.0 + 2.0 + 2.0) + nh * (16.0 + 12.0) + 100.0;
    // per atom: the Y contraction, 10 per Clebsch-Gordan term (complex product 6, scaled add 4)
    const double atom = 10.0 * s->T.total_terms;
    if (per_pair) *per_pair = pair;
    if (per_atom) *per_atom = atom;
    return PMD_OK;
}

int pmd_snap_reserve(pmd_snap* s, int nbatch, int natoms) {
    if (!s || nbatch < 0 || natoms < 0) return fail(PMD_EINVAL, "pmd_snap_reserve: bad arguments");
    return snap_reserve_impl(s, (long)nbatch * natoms);
}

int snap_energy_forces(pmd_snap* s, int nbatch, int natoms, const double box[3], const double* pos, const double* beta,
                       double* energy, double* forces, double* sumB, pmd_stream_t stream) {
    if (!s) return fail(PMD_EINVAL, "snap_energy_forces: NULL context");
    if (nbatch < 0 || natoms < 1) return fail(PMD_EINVAL, "snap_energy_forces: need nbatch >= 0 and natoms >= 1");
    int rc = check_box(box, s->p.rcut);
    if (rc) return rc;
    if (nbatch == 0) return PMD_OK;
    if (!pos || !beta) return fail(PMD_EINVAL, "snap_energy_forces: pos and beta are required");
    return snap_compute(s, nbatch, natoms, box, pos, beta, energy, forces, sumB, (cudaStream_t)stream);
}

int pmd_snap_sync_status(pmd_snap* s, pmd_stream_t stream) {
    if (!s) return fail(PMD_EINVAL, "pmd_snap_sync_status: NULL context");
    return read_status(s->s_status.as<int>(), (cudaStream_t)stream);
}

int eam_energy_forces(const pmd_fs_params* p, int nbatch, int natoms, const double box[3], const double* pos,
                      double* energy, double* forces, pmd_stream_t stream) {
    int rc = check_fs(p);
    if (rc) return rc;
    if (nbatch < 0 || natoms < 1) return fail(PMD_EINVAL, "eam_energy_forces: need nbatch >= 0 and natoms >= 1");
    if (natoms > PMD_MAX_COARSE_ATOMS) return fail(PMD_EUNSUPPORTED, "eam_energy_forces: natoms > PMD_MAX_COARSE_ATOMS");
    if ((rc = check_box(box, std::fmax(p->d, p->c)))) return rc;
    if (nbatch == 0) return PMD_OK;
    if (!pos) return fail(PMD_EINVAL, "eam_energy_forces: pos is NULL");
    return eam_launch(*p, nbatch, natoms, box, pos, energy, forces, (cudaStream_t)stream);
}

int pmd_engine_create(const pmd_engine_params* p, pmd_engine** out) {
    if (!out) return fail(PMD_EINVAL, "pmd_engine_create: out is NULL");
    *out = nullptr;
    if (!p) return fail(PMD_EINVAL, "pmd_engine_create: params are NULL");
    int rc;
    const bool csnap = p->coarse_kind == PMD_COARSE_SNAP;
    if (p->coarse_kind != PMD_COARSE_FS && !csnap) return fail(PMD_EINVAL, "pmd_engine_create: bad coarse_kind");
    if ((rc = check_snap_params(&p->fine)) || (rc = csnap ? check_snap_params(&p->coarse_snap) : check_fs(&p->coarse)))
        return rc;
    if (p->fine.twojmax > 8)
        return fail(PMD_EUNSUPPORTED, "pmd_engine_create: the fine propagator supports twojmax <= 8 "
                                      "(larger band limits: snap_energy_forces)");
    if (p->natoms < 1 || p->natoms > PMD_MAX_COARSE_ATOMS)
        return fail(PMD_EUNSUPPORTED, "pmd_engine_create: natoms must be in 1..PMD_MAX_COARSE_ATOMS");
    if (csnap && (p->coarse_snap.twojmax != 2 || p->natoms > 512))
        return fail(PMD_EUNSUPPORTED, "pmd_engine_create: a SNAP coarse potential needs twojmax = 2 and natoms <= 512");
    const double rc_coarse = csnap ? p->coarse_snap.rcut : std::fmax(p->coarse.d, p->coarse.c);
    if ((rc = check_box(p->box, std::fmax(p->fine.rcut, rc_coarse)))) return rc;
    pmd_engine* e = new (std::nothrow) pmd_engine();
    if (!e) return fail(PMD_ENOMEM, "pmd_engine_create: out of host memory");
    e->p = *p;
    cudaGetDevice(&e->device);
    cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
    if ((rc = pmd_snap_create(&p->fine, &e->snap))) {
        delete e;
        return rc;
    }
    if (csnap) {
        if ((rc = pmd_snap_create(&p->coarse_snap, &e->csnap)) ||
            (rc = e->cbeta.ensure((size_t)(1 + e->csnap->T.nB) * sizeof(double)))) {
            pmd_engine_destroy(e);
            return rc;
        }
        cudaError_t ce0 = cudaMemset(e->cbeta.p, 0, e->cbeta.bytes);
        if (ce0 != cudaSuccess) {
            pmd_engine_destroy(e);
            return cuda_fail(ce0, "pmd_engine_create");
        }
    }
    if ((rc = e->beta.ensure((size_t)(1 + e->snap->T.nB) * sizeof(double))) ||
        (rc = e->status.ensure(16 * sizeof(int))) || (rc = e->s_result.ensure(64))) {
        pmd_engine_destroy(e);
        return rc;
    }
    cudaError_t ce = cudaMemset(e->beta.p, 0, e->beta.bytes);
    if (ce == cudaSuccess) ce = cudaMemset(e->status.p, 0, e->status.bytes);
    if (ce == cudaSuccess) ce = cudaMallocHost(&e->pinned, 64);
    if (ce != cudaSuccess) {
        pmd_engine_destroy(e);
        return cuda_fail(ce, "pmd_engine_create");
    }
    *out = e;
    return PMD_OK;
}

int pmd_engine_destroy(pmd_engine* e) {
    if (!e) return PMD_OK;
    DevBuf* bufs[] = {&e->beta, &e->status, &e->s_nbr, &e->s_nnb, &e->s_dedr, &e->s_qf, &e->s_vh, &e->s_order,
                      &e->s_result, &e->s_noise, &e->s_gstep, &e->s_pos, &e->s_flow,
                      &e->s_selftest, &e->cbeta};
    for (DevBuf* b : bufs) b->release();
    if (e->pinned) cudaFreeHost(e->pinned);
    if (e->ev0) cudaEventDestroy(e->ev0);
    if (e->ev1) cudaEventDestroy(e->ev1);
    pmd_snap_destroy(e->snap);
    pmd_snap_destroy(e->csnap);
    delete e;
    return PMD_OK;
}

int pmd_engine_set_coarse_beta(pmd_engine* e, const double* beta, pmd_stream_t stream) {
    if (!e || !beta) return fail(PMD_EINVAL, "pmd_engine_set_coarse_beta: NULL argument");
    if (!e->csnap) return fail(PMD_EINVAL, "pmd_engine_set_coarse_beta: the engine's coarse potential is not SNAP");
    PMD_CUDA_TRY(cudaMemcpyAsync(e->cbeta.p, beta, e->cbeta.bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PMD_OK;
}

int pmd_engine_set_beta(pmd_engine* e, const double* beta, pmd_stream_t stream) {
    if (!e || !beta) return fail(PMD_EINVAL, "pmd_engine_set_beta: NULL argument");
    PMD_CUDA_TRY(cudaMemcpyAsync(e->beta.p, beta, e->beta.bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PMD_OK;
}

int pmd_engine_reserve(pmd_engine* e, int nbatch) {
    if (!e || nbatch < 0) return fail(PMD_EINVAL, "pmd_engine_reserve: bad arguments");
    if (nbatch <= e->cap_batch) return PMD_OK;
    const long na = (long)nbatch * e->p.natoms;
    const size_t rs = e->p.fine.precision == PMD_FP64 ? 8 : 4;
    int rc;
    if ((rc = e->s_nbr.ensure(na * PMD_MAX_NEIGHBORS * sizeof(int))) || (rc = e->s_nnb.ensure(na * sizeof(int))) ||
        (rc = e->s_dedr.ensure(na * PMD_MAX_NEIGHBORS * 3 * rs)) || (rc = e->s_qf.ensure(na * sizeof(float4))) ||
        (rc = e->s_vh.ensure(na * 3 * sizeof(double))) || (rc = e->s_order.ensure((2 * (size_t)nbatch + 4) * sizeof(int))) ||
        (rc = e->s_gstep.ensure(na * 3 * sizeof(double))) ||
        (rc = e->s_flow.ensure((2 * (size_t)nbatch + 2) * sizeof(unsigned long long))))
        return rc;
    if (e->p.natoms <= PMD_POS_TABLE_MAX_ATOMS && (rc = e->s_pos.ensure((size_t)na * e->p.natoms))) return rc;
    e->cap_batch = nbatch;
    return PMD_OK;
}

int pmd_engine_selftest_waits(pmd_engine* e, long long polls, pmd_stream_t stream) {
    if (!e || polls < 1) return fail(PMD_EINVAL, "pmd_engine_selftest_waits: need an engine and polls >= 1");
    return selftest_waits(e, polls, (cudaStream_t)stream);
}

int pmd_engine_profile(pmd_engine* e, int enable, double* last_ms) {
    if (!e) return fail(PMD_EINVAL, "pmd_engine_profile: NULL engine");
    if (enable && !e->ev0) {
        PMD_CUDA_TRY(cudaEventCreate(&e->ev0));
        PMD_CUDA_TRY(cudaEventCreate(&e->ev1));
    }
    if (last_ms) {
        *last_ms = -1.0;
        if (e->prof_recorded) {
            float ms = 0.f;
            PMD_CUDA_TRY(cudaEventSynchronize(e->ev1));
            PMD_CUDA_TRY(cudaEventElapsedTime(&ms, e->ev0, e->ev1));
            *last_ms = ms;
        }
    }
    e->profile = enable ? 1 : 0;
    return PMD_OK;
}

int pmd_sync_status(pmd_engine* e, pmd_stream_t stream) {
    if (!e) return fail(PMD_EINVAL, "pmd_sync_status: NULL engine");
    return read_status(e->status.as<int>(), (cudaStream_t)stream);
}

int baoab_propagate_batch(pmd_engine* e, int potential, int nbatch, int natoms, double* q, double* v,
                          int64_t member_stride, const int32_t* nsteps, const int64_t* interval_id,
                          const pmd_langevin* lp, pmd_stream_t stream) {
    if (!e) return fail(PMD_EINVAL, "baoab_propagate_batch: NULL engine");
    int rc = check_langevin(lp);
    if (rc) return rc;
    if (natoms != e->p.natoms) return fail(PMD_EINVAL, "baoab_propagate_batch: natoms differs from the engine's");
    if (nbatch < 0 || member_stride < 3L * natoms)
        return fail(PMD_EINVAL, "baoab_propagate_batch: need nbatch >= 0 and member_stride >= 3*natoms");
    if (nbatch == 0) return PMD_OK;
    if (!q || !v || !nsteps || !interval_id) return fail(PMD_EINVAL, "baoab_propagate_batch: NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    if (potential == PMD_FINE) {
        if ((rc = pmd_engine_reserve(e, nbatch))) return rc;
        return fine_propagate(e, nbatch, natoms, q, v, (long)member_stride, nsteps, interval_id, *lp, st);
    }
    if (potential == PMD_COARSE)
        return coarse_propagate(e, nbatch, natoms, q, v, (long)member_stride, nsteps, interval_id, *lp, st);
    return fail(PMD_EINVAL, "baoab_propagate_batch: potential must be PMD_FINE or PMD_COARSE");
}

int parareal_jumps(pmd_engine* e, int count, const double* fine_out, const double* coarse_prev, double* jumps,
                   pmd_stream_t stream) {
    if (!e || count < 0) return fail(PMD_EINVAL, "parareal_jumps: bad arguments");
    if (count == 0) return PMD_OK;
    if (!fine_out || !coarse_prev || !jumps) return fail(PMD_EINVAL, "parareal_jumps: NULL array");
    return jumps_launch((long)count * 6 * e->p.natoms, fine_out, coarse_prev, jumps, e->num_sms, (cudaStream_t)stream);
}

int parareal_correct(pmd_engine* e, int n_in, int n_fin, const double* jumps, const double* prev, double* cur,
                     double* coarse_out, double delta_expl, int metric, int L, const pmd_langevin* lp,
                     double* delta_host, int* n_stop_host, pmd_stream_t stream) {
    if (!e) return fail(PMD_EINVAL, "parareal_correct: NULL engine");
    int rc = check_langevin(lp);
    if (rc) return rc;
    if (n_in < 0 || n_fin < n_in || L < 0) return fail(PMD_EINVAL, "parareal_correct: need 0 <= n_in <= n_fin, L >= 0");
    if (lp->schedule == PMD_SCHED_L1_SYM && L > 1) return fail(PMD_EINVAL, "parareal_correct: L1_SYM needs L <= 1");
    if (metric != PMD_METRIC_REL && metric != PMD_METRIC_MAXDISP) return fail(PMD_EINVAL, "parareal_correct: bad metric");
    if (!prev || !cur || !coarse_out || !delta_host || !n_stop_host) return fail(PMD_EINVAL, "parareal_correct: NULL argument");
    if (std::isnan(delta_expl)) return fail(PMD_EINVAL, "parareal_correct: delta_expl is NaN");
    rc = parareal_sweep(e, n_in, n_fin, jumps, prev, cur, coarse_out, delta_expl, metric, L, *lp, delta_host,
                        n_stop_host, (cudaStream_t)stream);
    if (rc) return rc;
    return read_status(e->status.as<int>(), (cudaStream_t)stream);
}

}  // extern "C"
