/*
 * pmd_oracle.h -- the FP64 CPU oracle for the adaptive-parareal Langevin hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this library.  The product path (the CUDA
 * library under paper_2212_10508_gb300/) never calls it and shares no code, header,
 * table or constant generator with it.
 *
 * Every routine is a plain, slow, literal statement of what the paper (arXiv
 * 2212.10508) or the method it cites computes, in double precision:
 *   - Langevin scheme: eqs. (2)-(3) (Sec. 2), temperature-corrected form eqs. (11)-(12)
 *     with the schedules (13)-(14) (Sec. 2.4, App. A.2);
 *   - shared noise G_{l,n}: Sec. 2.1 and 2.3 (same Gaussian increments for F and C and
 *     every parareal iteration), drawn here from Philox4x32-10 + Box-Muller;
 *   - SNAP (Sec. 3.1, cited method of Thompson et al. 2015): bispectrum of the
 *     neighbour density on the 3-sphere, linear energy, forces by the chain rule;
 *   - EAM (Sec. 3.1, Finnis-Sinclair form with the tungsten constants of the workload).
 *
 * Units: metal (Angstrom, ps, eV, u, K).  Positions/velocities are SoA [batch][3][natoms].
 */
#ifndef PMD_ORACLE_H
#define PMD_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* physical constants (metal units) */
#define OR_KB 8.617333262e-5          /* eV/K */
#define OR_FTOA 9648.533215665        /* 1 eV/(Angstrom*u) in Angstrom/ps^2 */

typedef struct {
    int twojmax;      /* 2J: bispectrum band limit (8 for the 55-component SNAP) */
    double rcut;      /* cutoff radius, Angstrom */
    double rfac0;     /* theta0 = rfac0*pi*(r-rmin0)/(rcut-rmin0) */
    double rmin0;
    int switchflag;   /* 1: weight fc(r) = (cos(pi r/rcut)+1)/2 ; 0: weight 1 */
} or_snap_params;

typedef struct {      /* Finnis-Sinclair: rho=sum(r-d)^2 (r<d), V=(r-c)^2(c0+c1 r+c2 r^2) (r<c), F=-A sqrt(rho) */
    double d, A, c, c0, c1, c2;
} or_fs_params;

enum { OR_POT_SNAP = 0, OR_POT_FS = 1, OR_POT_ZERO = 2 };
enum { OR_SCHEME_PAPER = 0, OR_SCHEME_BAOAB = 1 };
enum { OR_SCHED_NONE = 0, OR_SCHED_ROBUST = 1, OR_SCHED_L1_SYM = 2 };

typedef struct {
    int kind;                 /* OR_POT_* */
    or_snap_params snap;
    const double* beta;       /* SNAP: [1+nB], beta[0] = per-atom constant */
    or_fs_params fs;
} or_potential;

typedef struct {
    double dt;        /* ps */
    double gamma;     /* 1/ps */
    double T;         /* K */
    double mass;      /* u */
    int scheme;       /* OR_SCHEME_* */
    int schedule;     /* OR_SCHED_* */
    uint64_t seed;    /* Philox key */
} or_langevin;

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The three standard normals G_{l,n} of one atom (x,y,z): counter (2*atom+blk, l, n_lo, n_hi). */
void or_normals3(uint64_t seed, int64_t n, int32_t ell, int32_t atom, double g[3]);

/* Clebsch-Gordan <j1 m1 j2 m2 | J M> by the Racah formula; all arguments doubled. */
double or_cg(int tj1, int tm1, int tj2, int tm2, int tJ, int tM);
/* Wigner U^j(a,b), 2j = tj, explicit polynomial formula; out[(p)*(tj+1)+q] = U_{m',m},
   p = j+m', q = j+m.  out is interleaved complex (re,im). */
void or_wigner_u(int tj, double are, double aim, double bre, double bim, double* out);

/* bispectrum index triples (2j1,2j2,2j) with j2<=j1<=j; returns count, fills out[3*count] if non-NULL */
int or_snap_triples(int twojmax, int* out);

/* SNAP energies/forces for nbatch independent periodic systems.
   energy[nbatch], forces[nbatch][3][natoms], sumB[nbatch][1+nB] (dE/dbeta; slot 0 = natoms),
   Bat[nbatch][natoms][nB] per-atom bispectrum; any output may be NULL.
   Returns 0, or -1 on bad arguments. */
int or_snap_energy_forces(const or_snap_params* p, int nbatch, int natoms, const double box[3],
                          const double* pos, const double* beta, double* energy, double* forces,
                          double* sumB, double* Bat);
int or_fs_energy_forces(const or_fs_params* p, int nbatch, int natoms, const double box[3],
                        const double* pos, double* energy, double* forces);
/* brute-force minimum-image neighbour lists, sorted by index; returns max count, -1 on overflow */
int or_neighbors(int natoms, const double* pos, const double box[3], double rc, int nmax,
                 int* cnt, int* list);

/* Propagate nbatch members, member b for nsteps[b] steps of the chosen scheme with
   interval id interval_id[b] as the noise key.  q, v in/out.  Returns 0 or -1. */
int or_propagate(const or_potential* pot, int nbatch, int natoms, const double box[3],
                 double* q, double* v, const int32_t* nsteps, const int64_t* interval_id,
                 const or_langevin* lp);

/* number of OpenMP threads the oracle uses */
int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
