/*
 * pmd.h -- C ABI of the GB300 (sm_103a) library for the hot path of adaptive parareal
 * Langevin dynamics with a SNAP fine potential and a Finnis-Sinclair EAM coarse
 * potential (Gorynina, Legoll, Lelievre, Perez, arXiv 2212.10508).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status (PMD_OK = 0, negative on error).  pmd_last_error()
 *    returns a thread-local, NUL-terminated message describing the last failure.
 *  - Array arguments are caller-owned DEVICE pointers unless marked "host".  The library
 *    never frees or retains them past the call.  No allocation or exception crosses the ABI.
 *  - Positions q, velocities v and forces are FP64, structure-of-arrays per system:
 *    [member][3][natoms] (x row, y row, z row).  Positions are unwrapped Angstrom; the box
 *    is orthorhombic and periodic (minimum image), box[3] = edge lengths (host array).
 *    Every box edge must exceed twice the largest cutoff used.
 *  - Units: Angstrom, ps, eV, u (atomic mass), K.
 *  - Calls that take a stream enqueue their kernels on it and return without
 *    synchronising, unless documented otherwise.  Errors found on the device (neighbour
 *    capacity, non-finite state, a wait that timed out) are recorded in the context's
 *    status word and reported by pmd_sync_status() and by every call that synchronises.
 *  - Contexts (pmd_snap, pmd_engine) own their device tables, scratch and status word.
 *    A context may be used by one host thread at a time.  Scratch grows on demand with
 *    cudaMalloc; call the *_reserve() functions before capturing calls into a CUDA graph.
 */
#ifndef PMD_H
#define PMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* pmd_stream_t;   /* a cudaStream_t; NULL selects the legacy default stream */

enum {
    PMD_OK = 0,
    PMD_EINVAL = -1,        /* bad argument (sizes, NULL pointers, parameter ranges) */
    PMD_ENOMEM = -2,        /* device or pinned allocation failed */
    PMD_ECUDA = -3,         /* a CUDA runtime call failed (message in pmd_last_error) */
    PMD_ENEIGH = -4,        /* an atom had more neighbours than PMD_MAX_NEIGHBORS */
    PMD_ENONFINITE = -5,    /* a position or velocity became NaN or infinite */
    PMD_ETIMEOUT = -6,      /* a bounded device-side wait gave up (the call's output is invalid) */
    PMD_ELOSTATOM = -7,     /* an atom moved more than half a box edge in one step */
    PMD_EUNSUPPORTED = -8   /* valid request this build does not support (e.g. size limits) */
};

#define PMD_MAX_NEIGHBORS 64      /* per-atom neighbour capacity of the SNAP and EAM kernels */
#define PMD_MAX_TWOJMAX 14        /* largest 2J the SNAP kernels are built for (2J > 8: FP64 and
                                     snap_energy_forces only; 14 is the paper's SNAP-205) */
#define PMD_MAX_COARSE_ATOMS 2048 /* largest system the one-CTA coarse propagator accepts */

enum { PMD_FP64 = 0, PMD_FP32_BULK = 1 };            /* arithmetic of the potential kernels */
enum { PMD_FINE = 0, PMD_COARSE = 1 };               /* which potential drives a propagation */
enum { PMD_SCHEME_PAPER = 0, PMD_SCHEME_BAOAB = 1 }; /* Langevin integrator */
enum { PMD_SCHED_NONE = 0, PMD_SCHED_ROBUST = 1, PMD_SCHED_L1_SYM = 2 };
enum { PMD_METRIC_REL = 0, PMD_METRIC_MAXDISP = 1 };

/* ------------------------------------------------------------------------------------
 * Parameters
 * ---------------------------------------------------------------------------------- */

/* SNAP (Sec. 3.1; the fine potential V_F; method of Thompson et al. 2015, which the paper
 * cites).  Neighbour k of atom i at r < rcut maps to the unit quaternion
 * a = cos(t0) - i sin(t0) z/r, b = sin(t0)(y - i x)/r with t0 = rfac0*pi*r/rcut; the
 * bispectrum B_{j1 j2 j} (0 <= j2 <= j1 <= j <= twojmax/2) of the weighted density
 * I + sum_k fc(r_k) U(a_k, b_k), fc = (cos(pi r/rcut)+1)/2, enters E_i = beta_0 + sum_t beta_t B_t. */
typedef struct {
    int twojmax;      /* 2J, even, 2..PMD_MAX_TWOJMAX (8 gives the 55 components of SNAP-56, 14 the
                         204 of SNAP-205); above 8 FP64 only, and no engine (propagation) */
    double rcut;      /* Angstrom */
    double rfac0;     /* in (0, 1] */
    double rmin0;     /* must be 0 */
    int switchflag;   /* 1: weights fc(r); 0: weights 1 */
    int precision;    /* PMD_FP64, or PMD_FP32_BULK: U/Z/Y arithmetic in FP32 (the bispectrum's
                         Z elements included), the bispectrum's sum over elements and the force
                         sums in double-float (FP64-class), energy sums in FP64 */
} pmd_snap_params;

/* Finnis-Sinclair EAM (Sec. 3.1; the coarse potential V_C):
 * rho_i = sum_{r<d}(r-d)^2, E = sum_i -A sqrt(rho_i) + 1/2 sum_{i!=j, r<c}(r-c)^2(c0+c1 r+c2 r^2). */
typedef struct {
    double d, A, c, c0, c1, c2;
    int precision;    /* PMD_FP64 or PMD_FP32_BULK (pair terms in FP32, sums in FP64) */
} pmd_fs_params;

/* Langevin integrator (Sec. 2, eqs. (2)-(3); with a temperature schedule eqs. (11)-(14)).
 * PAPER: per sub-step l, with a(q) = F(q)/m, kT = k_B T / m, C_l the schedule:
 *   v_{l+1/2} = v_l + dt/2 a(q_l) - dt/2 gamma v_{l-1/2} + 1/2 sqrt(2 gamma kT C_l dt) G_l
 *   q_{l+1}   = q_l + dt v_{l+1/2}
 *   v_{l+1}   = v_{l+1/2} + dt/2 a(q_{l+1}) - dt/2 gamma v_{l+1/2} + 1/2 sqrt(2 gamma kT C_{l+1} dt) G_{l+1}
 * with v_{-1/2} := v_0; each call restarts at l = 0 (one parareal interval).
 * BAOAB: Leimkuhler-Matthews splitting with the exact Ornstein-Uhlenbeck step.
 * Noise G_{l,n}: Philox4x32-10 keyed by seed, counter (2*atom+blk, l, n_lo, n_hi), Box-Muller
 * on 53-bit uniforms; identical for fine and coarse and every parareal iteration (Sec. 2.1). */
typedef struct {
    double dt;        /* ps */
    double gamma;     /* 1/ps, >= 0 */
    double T;         /* K, >= 0 */
    double mass;      /* u, > 0 */
    int scheme;       /* PMD_SCHEME_PAPER or PMD_SCHEME_BAOAB */
    int schedule;     /* PMD_SCHED_NONE (C_l = 1), ROBUST (C_0 = 3, C_l = 1, eq. (13)),
                         L1_SYM (C_0 = C_1 = 2, eq. (14); every nsteps must be <= 1) */
    uint64_t seed;    /* Philox key */
} pmd_langevin;

/* ------------------------------------------------------------------------------------
 * Errors
 * ---------------------------------------------------------------------------------- */

/* Message of the last failed call on this host thread (never NULL). */
const char* pmd_last_error(void);

/* ------------------------------------------------------------------------------------
 * SNAP context and energies/forces
 * ---------------------------------------------------------------------------------- */
typedef struct pmd_snap pmd_snap;

/* Builds the Clebsch-Gordan and contraction tables on the current CUDA device.
 * *out receives an owned context (free with pmd_snap_destroy).  EINVAL on bad parameters. */
int pmd_snap_create(const pmd_snap_params* p, pmd_snap** out);
int pmd_snap_destroy(pmd_snap* s);
/* Number of coefficients 1 + nB (beta_0 plus one per bispectrum component). */
int pmd_snap_num_coeffs(const pmd_snap* s);
/* Grow the context's scratch for nbatch*natoms atoms now (no allocation happens later in
 * calls that stay within this size). */
int pmd_snap_reserve(pmd_snap* s, int nbatch, int natoms);

/* Algorithmic FP operation counts of the SNAP force kernels, enumerated from the context's own
 * tables (half-layout recursion, contraction jobs, force contraction): *per_pair = operations per
 * neighbour pair (U recursion and accumulation, plus the dE/dr pass), *per_atom = operations per
 * atom independent of its neighbour count (the Y contraction).  A complex multiply counts 6, a
 * real fused multiply-add 2.  Used for roofline accounting; any pointer may be NULL. */
int pmd_snap_flop_model(const pmd_snap* s, double* per_pair, double* per_atom);

/* Measured FMA throughput of the current device, the denominator of the ALU roofline of the
 * SNAP kernels (a microbenchmark; the paper has no counterpart).  kind: PMD_PEAK_FFMA (scalar
 * FP32 fmaf), PMD_PEAK_FFMA2 (paired FP32 __ffma2_rn, the form the batched contraction uses) or
 * PMD_PEAK_DFMA (FP64 fma).  Every SM is filled with 2048 threads running 16 (FP32) or 8 (FP64)
 * independent FMA chains each; a short launch sizes one timed launch of about `seconds`
 * (0 < seconds <= 10) on `stream`, timed with CUDA events.  *tflops = 2 x FMAs / time in
 * TFLOP/s; *ms (may be NULL) the timed launch's duration.  Synchronises the stream. */
enum { PMD_PEAK_FFMA = 0, PMD_PEAK_FFMA2 = 1, PMD_PEAK_DFMA = 2 };
int pmd_alu_peak(int kind, double seconds, pmd_stream_t stream, double* tflops, double* ms);

/* SNAP energies and forces of nbatch independent systems (Sec. 3.1).
 *   pos    [nbatch][3][natoms]  FP64 device, unwrapped Angstrom
 *   beta   [1+nB]               FP64 device, beta[0] = per-atom constant
 *   energy [nbatch]             FP64 device or NULL: E = sum_i E_i (eV)
 *   forces [nbatch][3][natoms]  FP64 device or NULL: F = -dE/dq (eV/Angstrom)
 *   sumB   [nbatch][1+nB]       FP64 device or NULL: dE/dbeta (sumB[0] = natoms, sumB[1+t] = sum_i B_t)
 * With forces == NULL only the U_tot and bispectrum stages run (no adjoint, no dE/dr pass).
 * Stream-ordered; ENEIGH/ENONFINITE surface at pmd_snap_sync_status. */
int snap_energy_forces(pmd_snap* s, int nbatch, int natoms, const double box[3], const double* pos,
                       const double* beta, double* energy, double* forces, double* sumB,
                       pmd_stream_t stream);
/* Synchronises the stream and returns (and clears) the context's device status. */
int pmd_snap_sync_status(pmd_snap* s, pmd_stream_t stream);

/* The same energies, forces and dE/dbeta as snap_energy_forces, for callers that may not
 * allocate device memory while they run (an application that owns all device memory through
 * its own allocator, a loop where cudaMalloc would stall or is not allowed, a fixed memory
 * budget).  The paper has no counterpart; it is an interface addition of this library.
 * Scratch comes from one array of PMD_NOALLOC_SCRATCH_BYTES compiled into the library.
 * pmd_snap_create loads that array on its device (with lazy module loading, the CUDA default,
 * this is when its 16 MiB are reserved), and the device keeps it until the process exits; the
 * call itself allocates nothing.  The context s must exist already (its tables are allocated
 * by pmd_snap_create) and must belong to the current device.  Each call looks up the array's
 * address in the current context.  All calls on a device share the array and find the last
 * call's contents there: calls whose kernels overlap on the GPU race on it.  Box and argument
 * checks are those of snap_energy_forces.  Requests whose scratch exceeds the array (about
 * 1 KiB per atom for FP32 forces, 3.7 KiB with energies; twice that in FP64) return
 * PMD_EUNSUPPORTED. */
#define PMD_NOALLOC_SCRATCH_BYTES (16u << 20)
int snap_energy_forces_noalloc(pmd_snap* s, int nbatch, int natoms, const double box[3], const double* pos,
                               const double* beta, double* energy, double* forces, double* sumB,
                               pmd_stream_t stream);

/* Finnis-Sinclair EAM energies and forces of nbatch systems (Sec. 3.1), one CTA per system,
 * no scratch.  energy [nbatch] and forces [nbatch][3][natoms] may each be NULL.
 * natoms <= PMD_MAX_COARSE_ATOMS (EUNSUPPORTED otherwise). */
int eam_energy_forces(const pmd_fs_params* p, int nbatch, int natoms, const double box[3],
                      const double* pos, double* energy, double* forces, pmd_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Engine: one fine (SNAP) and one coarse (EAM) potential on one periodic cell
 * ---------------------------------------------------------------------------------- */
typedef struct pmd_engine pmd_engine;

/* Coarse potential of an engine: Finnis-Sinclair EAM (Strategy II of Sec. 3, the default), or
 * SNAP with 2J = 2 (SNAP-6, Strategy I of Sec. 3; coefficients set by pmd_engine_set_coarse_beta). */
enum { PMD_COARSE_FS = 0, PMD_COARSE_SNAP = 1 };

typedef struct {
    pmd_snap_params fine;   /* fine potential V_F */
    pmd_fs_params coarse;   /* coarse potential V_C when coarse_kind = PMD_COARSE_FS */
    double box[3];          /* Angstrom */
    int natoms;             /* atoms per system */
    int coarse_kind;        /* PMD_COARSE_FS (0) or PMD_COARSE_SNAP */
    pmd_snap_params coarse_snap;   /* V_C when coarse_kind = PMD_COARSE_SNAP: twojmax must be 2,
                                      natoms <= 512 (EUNSUPPORTED otherwise) */
} pmd_engine_params;

int pmd_engine_create(const pmd_engine_params* p, pmd_engine** out);
int pmd_engine_destroy(pmd_engine* e);
/* Copy the SNAP coefficients beta [1+nB] (device pointer) into the engine (stream-ordered). */
int pmd_engine_set_beta(pmd_engine* e, const double* beta, pmd_stream_t stream);
/* Copy the coefficients beta [1 + 5] (device pointer, beta[0] = beta_0) of a SNAP coarse
 * potential (PMD_COARSE_SNAP) into the engine (stream-ordered); EINVAL for an EAM coarse
 * potential.  They start at zero. */
int pmd_engine_set_coarse_beta(pmd_engine* e, const double* beta, pmd_stream_t stream);
/* Grow the engine's scratch for batches of up to nbatch systems. */
int pmd_engine_reserve(pmd_engine* e, int nbatch);
/* Synchronises the stream and returns (and clears) the engine's device status. */
int pmd_sync_status(pmd_engine* e, pmd_stream_t stream);

/* Kernel timing hook for roofline accounting: while enabled, every FINE propagation records
 * CUDA events around its persistent kernel on the call's stream.  *last_ms (may be NULL)
 * receives the duration of the most recent such kernel (waits for it to finish), or -1 if none. */
int pmd_engine_profile(pmd_engine* e, int enable, double* last_ms);

/* Self-test of the bounded cross-CTA waits (failure detection without a GPU fault): launches one
 * CTA that waits on counters nothing increments (64-bit, as in the fine kernel's dataflow
 * schedule, and 32-bit) and then on a two-CTA grid barrier with only itself launched (the barrier
 * of the FP64 path), each for at most `polls` polls (>= 1; ~200 ns each).  All give up, and the
 * next pmd_sync_status returns PMD_ETIMEOUT; the engine stays usable.  EINVAL for polls < 1. */
int pmd_engine_selftest_waits(pmd_engine* e, long long polls, pmd_stream_t stream);

/* Run-time shape of the batched FP32 fine kernel (the FP64 form ignores it):
 *   rows2_atoms  batches of at most this many atoms (0..16) run the Y contraction with two output
 *                rows per warp (half-warps of 16 atoms), rows4_atoms (0..8) with four rows per warp;
 *   b_group      atoms per warp in the integrator phase (1..10);
 *   noise_stage  Y stage (by sub-block size tb, 0 = tb <= 3) that also draws the Gaussian
 *                increments of the batch, -1 = the stage of tb = 6;
 *   warps        warps per CTA of the persistent kernel, 16 (up to 128 registers per thread) or
 *                8 (up to 255: no register spills, half the warps to hide latency); 8 is built
 *                for 2J = 8 only, other band limits run with 16.
 * Results do not depend on the shape (every output keeps its arithmetic and order); only time
 * does.  Defaults {16, 8, 8, -1, 16}. */
typedef struct {
    int rows2_atoms, rows4_atoms, b_group, noise_stage, warps;
} pmd_fine_tuning;
int pmd_engine_get_tuning(const pmd_engine* e, pmd_fine_tuning* out);
int pmd_engine_set_tuning(pmd_engine* e, const pmd_fine_tuning* t);

/* Autotuner of the batched FP32 fine kernel: times baoab_propagate_batch(PMD_FINE) on a copy of
 * the given batch (q, v, member_stride, nsteps, interval_id, lp as in baoab_propagate_batch;
 * the caller's arrays are not modified) with the interval lengths scaled down so that the
 * longest takes max_steps steps (the shape of the active set over the sub-steps is kept), for a
 * set of candidate shapes (coordinate search, two timed runs each), and keeps the fastest in the
 * engine.  *chosen and *best_ms (each may be NULL) receive it and its time.  Setup call: it
 * allocates device memory and synchronises the stream.  EUNSUPPORTED for an FP64 fine engine. */
int pmd_engine_autotune(pmd_engine* e, int nbatch, int natoms, const double* q, const double* v,
                        int64_t member_stride, const int32_t* nsteps, const int64_t* interval_id,
                        const pmd_langevin* lp, int max_steps, pmd_stream_t stream, pmd_fine_tuning* chosen,
                        double* best_ms);

/* Propagate nbatch independent systems, member b for nsteps[b] steps of the Langevin scheme
 * lp driven by the fine (PMD_FINE, SNAP) or coarse (PMD_COARSE, EAM) potential, with noise
 * key n = interval_id[b]: member b computes F_dt or C_dt of the interval [n dt*L, ...]
 * (Sec. 2.1; all intervals of Algorithm 1/2's parallel step at once).
 *   q, v          device FP64, in/out; member b's positions start at q + b*member_stride,
 *                 rows x,y,z of length natoms (member_stride >= 3*natoms; 3*natoms for
 *                 [nbatch][3][natoms] arrays, 6*natoms to work inside packed states)
 *   nsteps        [nbatch] int32 device, 0 <= nsteps[b]
 *   interval_id   [nbatch] int64 device
 * FINE runs as one persistent cooperative kernel over all members: FP32_BULK as a dataflow
 * schedule (each member's sub-steps wait only on that member's own work), FP64 with per-step
 * grid barriers; every wait is bounded (ETIMEOUT at pmd_sync_status if one gives up).  The
 * results do not depend on the batch composition: a member gives the same bits alone or in any
 * batch.  COARSE runs one CTA per member.
 * natoms must equal the engine's natoms.  Stream-ordered. */
int baoab_propagate_batch(pmd_engine* e, int potential, int nbatch, int natoms, double* q, double* v,
                          int64_t member_stride, const int32_t* nsteps, const int64_t* interval_id,
                          const pmd_langevin* lp, pmd_stream_t stream);

/* Jumps of Algorithm 1/2 (Sec. 2.1, eq. (5)): J_n = F_dt(prev_n) - C_dt(prev_n), elementwise
 * over count packed states [count][6][natoms] (q rows then v rows).  Stream-ordered. */
int parareal_jumps(pmd_engine* e, int count, const double* fine_out, const double* coarse_prev,
                   double* jumps, pmd_stream_t stream);

/* The sequential correction sweep of Algorithm 2 (Sec. 2.2), on the coarse potential:
 * for n = n_in .. n_fin-1:
 *     coarse_out[n-n_in] = C_dt(cur_n)               (L steps, noise key n)
 *     cur_{n+1}          = coarse_out[n-n_in] + J_n
 *     delta              = E(prev, cur, n_in, n+1)    (metric below)
 *     if delta > delta_expl: *n_stop_host = n; stop   (Algorithm 2's "N_final := n")
 * States are packed [.][6][natoms] (q rows then v rows), device FP64:
 *   jumps [n_fin-n_in], prev [n_fin-n_in+1], cur [n_fin-n_in+1] (cur[0] = cur_{n_in} is read,
 *   the rest written), coarse_out [n_fin-n_in] (C_dt(cur_n), the C_dt(prev_n) of the next
 *   iteration).  jumps may be NULL (J = 0: the coarse initialisation of a new slab).
 * metric PMD_METRIC_REL: E = sum |q^cur_n - q^prev_n| / sum |q^prev_n| over n_in..n+1 with
 *   |.| the Euclidean norm of the 3m positions; PMD_METRIC_MAXDISP: the largest per-atom
 *   displacement |q_i^cur - q_i^prev| (Angstrom) over the same range.  A non-finite state
 *   counts as delta = +inf.
 * delta_host, n_stop_host: host outputs; *n_stop_host = n_fin when the sweep completes.
 * Execution: with the Finnis-Sinclair coarse potential and 64 <= natoms <= 512 the sweep runs on
 * one thread-block cluster of min(8, ceil(natoms/32)) CTAs (the atoms of each interval spread
 * over its SMs); otherwise on one CTA.  Either way coarse_out equals, bit for bit, what
 * baoab_propagate_batch(COARSE) computes from the same states.
 * This call SYNCHRONISES the stream (its outputs decide the host's next step).
 * L = steps per interval; lp as in baoab_propagate_batch. */
int parareal_correct(pmd_engine* e, int n_in, int n_fin, const double* jumps, const double* prev,
                     double* cur, double* coarse_out, double delta_expl, int metric, int L,
                     const pmd_langevin* lp, double* delta_host, int* n_stop_host, pmd_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Adaptive restart: the host state machine of Algorithm 2 (Sec. 2.2) and the cost model
 * of eqs. (7)-(9).  Pure host code; no device work.
 * ---------------------------------------------------------------------------------- */
typedef struct pmd_adaptive pmd_adaptive;

enum { PMD_ACT_ITERATE = 0, PMD_ACT_DONE = 1 };

typedef struct {
    int kind;        /* PMD_ACT_ITERATE or PMD_ACT_DONE */
    int n_in;        /* current slab [n_in, n_fin] */
    int n_fin;
    int open_slab;   /* 1: a new slab starts at n_in: run the coarse initialisation
                        cur_{n+1} = C(cur_n) over it (parareal_correct with jumps = NULL) first */
    int k;           /* iterations done so far on this slab (k^{N_slab}_conv) */
} pmd_action;

/* N: horizon in intervals; 0 < delta_conv < delta_expl. */
int pmd_adaptive_create(int N, double delta_conv, double delta_expl, pmd_adaptive** out);
int pmd_adaptive_destroy(pmd_adaptive* st);
/* Advance Algorithm 2.  The first call (delta and n_stop ignored) returns the first slab.
 * Every later call reports the result of the iteration just run -- delta and n_stop as
 * returned by parareal_correct -- and receives the next action.  When the explosion test
 * fires at n_stop = n_in the slab would be empty; it is shortened to [n_in, n_in+1] instead. */
int adaptive_restart(pmd_adaptive* st, double delta, int n_stop, pmd_action* next);
/* eqs. (7)-(9) over the run so far: Cost, Gamma_adapt = N C_f / Cost, Gamma_ideal = N / sum k.
 * Any output pointer may be NULL. */
int pmd_adaptive_cost(const pmd_adaptive* st, double C_f, double C_c, double* cost, double* gamma_adapt,
                      double* gamma_ideal);
/* Window log: number of (slab, end point) entries; entry i gives N_init^s, N_final^{s,j},
 * k^{s,j} and the slab index s (0-based).  Returns the count, or < 0 on error. */
int pmd_adaptive_log(const pmd_adaptive* st, int capacity, int* n_init, int* n_final, int* k, int* slab);

/* ---- SIA tracking (Sec. 3: location of the self-interstitial and its residence times) --------
 * The paper locates the interstitial by a Voronoi analysis of each frame and reports residence
 * times in a well in units of the time step (Sec. 3, the table of residence times, and the
 * statistical study that follows it).  Reading used here (Wigner-Seitz): every atom belongs to
 * its nearest site of a reference lattice shifted by the centre-of-mass displacement of the
 * frame; the interstitial's well is the site with the largest occupancy (2 for one interstitial;
 * the smallest site index on ties).
 *
 * sia_locate: frame f of `frames` starts at frames + f * frame_stride (doubles; >= 3 natoms) and
 * holds unwrapped positions [3][natoms] in Angstrom (so the states [N+1][6][natoms] of a parareal
 * run are frames with stride 6 natoms).  ref [3][natoms] are the positions the centre-of-mass
 * displacement is taken from (usually frame 0), sites [3][nsites] the reference lattice (device
 * pointers); box [3] is host memory.  Per frame, in FP64 with this rounding order (the same in any
 * implementation, so that every nearest-site decision is reproducible bit for bit):
 *   c_a   = (sum over i in index order of (q_ai - ref_ai)) / natoms          for a = x, y, z
 *   d_a   = ((q_ai - c_a) - s_a), then d_a -= L_a * rint(d_a / L_a)
 *   r2    = (d_x d_x + d_y d_y) + d_z d_z, no fused multiply-adds
 *   site  = the smallest index with the smallest r2.
 * Outputs (device, [nframes] int32): well[f] and occupancy[f] = the number of atoms on that site.
 * Asynchronous on `stream`.  EINVAL: nframes < 0, natoms < 1, nsites < 1 or > 4096, a NULL array
 * (when nframes > 0), frame_stride < 3 natoms, or a non-positive box length. */
int sia_locate(int nframes, int natoms, int nsites, const double box[3], const double* frames,
               int64_t frame_stride, const double* ref, const double* sites, int32_t* well,
               int32_t* occupancy, pmd_stream_t stream);

/* Residence times of a well sequence (host arrays): the lengths, in frames, of the runs of equal
 * consecutive wells, in order; the last run is still open at the end of the sequence and is not
 * returned (its length is a lower bound).  lengths and sites (may be NULL) receive at most
 * `capacity` entries; *nruns the number of completed runs.  EINVAL for NULL well / nruns or
 * nframes < 0; ENOMEM (nothing written beyond capacity) if capacity is too small. */
int sia_residence(const int32_t* well, int nframes, int capacity, int32_t* lengths, int32_t* sites, int* nruns);

#ifdef __cplusplus
}
#endif
#endif /* PMD_H */
