/*
 * pmd_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see pmd_oracle.h).
 *
 * Nothing here is blocked, fused or reordered for speed beyond caching Clebsch-Gordan
 * values per call.  Parallelism is plain OpenMP over independent atoms or systems.
 */
#include "pmd_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_in_parallel(void) { return 0; }
#endif

typedef double complex cplx;

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------
 * Noise.  The paper requires the same standard Gaussians G_{l,n} (0<=l<=L) for the
 * fine and the coarse propagator and at every parareal iteration (Sec. 2.1, where the two
 * propagators of one interval are driven by identical random increments; Sec. 2.3, seeds
 * S_n per interval).  They are drawn here from a counter-based generator:
 * Philox4x32-10 as published by Salmon et al. (SC'11): 10 rounds of
 *   (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))
 * with M0=0xD2511F53, M1=0xCD9E8D57 and the key bumped by (0x9E3779B9, 0xBB67AE85)
 * between rounds.
 * ---------------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller on two 53-bit uniforms built from one Philox block:
   U1 = ((x0>>5)*2^26 + (x1>>6)) * 2^-53 in [0,1), u1 = 1-U1 in (0,1];
   u2 = ((x2>>5)*2^26 + (x3>>6)) * 2^-53 in [0,1);
   (g_a, g_b) = sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2). */
static void box_muller(const uint32_t x[4], double* ga, double* gb) {
    const double two_m53 = 1.0 / 9007199254740992.0;
    double U1 = (double)(((uint64_t)(x[0] >> 5) << 26) | (uint64_t)(x[1] >> 6)) * two_m53;
    double u2 = (double)(((uint64_t)(x[2] >> 5) << 26) | (uint64_t)(x[3] >> 6)) * two_m53;
    double u1 = 1.0 - U1;
    double R = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    *ga = R * cos(ang);
    *gb = R * sin(ang);
}

/* G_{l,n} for one atom: key = (seed_lo, seed_hi); counter = (2*atom+blk, l, n_lo, n_hi);
   block 0 -> (G_x, G_y), block 1 -> G_z (its sine partner is unused). */
void or_normals3(uint64_t seed, int64_t n, int32_t ell, int32_t atom, double g[3]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t un = (uint64_t)n;
    uint32_t ctr[4], x[4];
    double unused;
    ctr[0] = 2u * (uint32_t)atom;
    ctr[1] = (uint32_t)ell;
    ctr[2] = (uint32_t)un;
    ctr[3] = (uint32_t)(un >> 32);
    or_philox4x32_10(ctr, key, x);
    box_muller(x, &g[0], &g[1]);
    ctr[0] = 2u * (uint32_t)atom + 1u;
    or_philox4x32_10(ctr, key, x);
    box_muller(x, &g[2], &unused);
}

/* ------------------------------------------------------------------------------------
 * Clebsch-Gordan coefficients by the Racah formula (Condon-Shortley phases).
 * Arguments are doubled (tj = 2j, tm = 2m).
 * ---------------------------------------------------------------------------------- */
static double fact(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= (double)k;
    return f;
}

double or_cg(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
    if (tm1 + tm2 != tM) return 0.0;
    if (abs(tm1) > tj1 || abs(tm2) > tj2 || abs(tM) > tJ) return 0.0;
    if (((tj1 + tm1) & 1) || ((tj2 + tm2) & 1) || ((tJ + tM) & 1)) return 0.0;
    if (tJ < abs(tj1 - tj2) || tJ > tj1 + tj2 || ((tj1 + tj2 + tJ) & 1)) return 0.0;
    /* integer combinations */
    int J_j1_j2 = (tJ + tj1 - tj2) / 2;   /* J + j1 - j2 */
    int J_j2_j1 = (tJ - tj1 + tj2) / 2;   /* J - j1 + j2 */
    int j1_j2_J = (tj1 + tj2 - tJ) / 2;   /* j1 + j2 - J */
    int all1 = (tj1 + tj2 + tJ) / 2 + 1;  /* j1 + j2 + J + 1 */
    int JpM = (tJ + tM) / 2, JmM = (tJ - tM) / 2;
    int j1m1m = (tj1 - tm1) / 2, j1m1p = (tj1 + tm1) / 2;
    int j2m2m = (tj2 - tm2) / 2, j2m2p = (tj2 + tm2) / 2;
    double pre = sqrt((tJ + 1) * fact(J_j1_j2) * fact(J_j2_j1) * fact(j1_j2_J) / fact(all1));
    pre *= sqrt(fact(JpM) * fact(JmM) * fact(j1m1m) * fact(j1m1p) * fact(j2m2m) * fact(j2m2p));
    double sum = 0.0;
    for (int k = 0; k <= all1; ++k) {
        int d1 = j1_j2_J - k;
        int d2 = j1m1m - k;
        int d3 = j2m2p - k;
        int d4 = (tJ - tj2 + tm1) / 2 + k;  /* J - j2 + m1 + k */
        int d5 = (tJ - tj1 - tm2) / 2 + k;  /* J - j1 - m2 + k */
        if (d1 < 0 || d2 < 0 || d3 < 0 || d4 < 0 || d5 < 0) continue;
        double den = fact(k) * fact(d1) * fact(d2) * fact(d3) * fact(d4) * fact(d5);
        sum += ((k & 1) ? -1.0 : 1.0) / den;
    }
    return pre * sum;
}

/* ------------------------------------------------------------------------------------
 * SNAP.  The paper defines SNAP by citation only (Thompson et al. 2015).  Reading:
 * each neighbour k of atom i at distance r < rcut is mapped to the unit quaternion
 *   a = cos(theta0) - i sin(theta0) z/r,  b = sin(theta0) (y - i x)/r,
 *   theta0 = rfac0 * pi * r / rcut,
 * i.e. the SU(2) element g = [[a, b], [-conj b, conj a]].  U^j(g) is the spin-j
 * representation in the |j m> basis, written here by the explicit polynomial formula
 * obtained from the action of g on homogeneous polynomials x^(j+m) y^(j-m):
 *   U^j_{m',m} = sqrt((j+m')!(j-m')!/((j+m)!(j-m)!))
 *       * sum_s C(j+m,s) C(j-m,j-m'-s) a^(j+m-s) conj(a)^(j-m'-s) b^(m'-m+s) (-conj b)^s.
 * U_tot^j = I + sum_k fc(r_k) U^j(g_k);  B_{j1 j2 j} = Re sum conj(U_tot^j)_{m m'}
 *   sum C^{jm}_{j1 m1 j2 m2} C^{jm'}_{j1 m1' j2 m2'} (U_tot^{j1})_{m1 m1'} (U_tot^{j2})_{m2 m2'};
 * E_i = beta_0 + sum_t beta_t B_t.
 * ---------------------------------------------------------------------------------- */
static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    return fact(n) / (fact(k) * fact(n - k));
}

/* U^j and its Wirtinger partials d/da, d/d(conj a), d/db, d/d(conj b); any of the
   partial outputs may be NULL.  Layout [p][q], p = j+m', q = j+m. */
static void wigner_u_partials(int tj, cplx a, cplx b, cplx* U, cplx* Ua, cplx* Uac, cplx* Ub,
                              cplx* Ubc) {
    int n = tj + 1;
    cplx ac = conj(a), mbc = -conj(b);
    cplx pa[32], pac[32], pb[32], pmbc[32];
    pa[0] = pac[0] = pb[0] = pmbc[0] = 1.0;
    for (int k = 1; k <= tj; ++k) {
        pa[k] = pa[k - 1] * a;
        pac[k] = pac[k - 1] * ac;
        pb[k] = pb[k - 1] * b;
        pmbc[k] = pmbc[k - 1] * mbc;
    }
    for (int p = 0; p < n; ++p) {
        for (int q = 0; q < n; ++q) {
            double norm = sqrt(fact(p) * fact(tj - p) / (fact(q) * fact(tj - q)));
            cplx u = 0, ua = 0, uac = 0, ub = 0, ubc = 0;
            int s_lo = q - p > 0 ? q - p : 0;
            int s_hi = q < tj - p ? q : tj - p;
            for (int s = s_lo; s <= s_hi; ++s) {
                double cf = binom(q, s) * binom(tj - q, tj - p - s);
                int ea = q - s, eac = tj - p - s, eb = p - q + s, ebc = s;
                u += cf * pa[ea] * pac[eac] * pb[eb] * pmbc[ebc];
                if (ea > 0) ua += cf * ea * pa[ea - 1] * pac[eac] * pb[eb] * pmbc[ebc];
                if (eac > 0) uac += cf * eac * pa[ea] * pac[eac - 1] * pb[eb] * pmbc[ebc];
                if (eb > 0) ub += cf * eb * pa[ea] * pac[eac] * pb[eb - 1] * pmbc[ebc];
                /* d(-conj b)^s / d(conj b) = -s (-conj b)^(s-1) */
                if (ebc > 0) ubc += -cf * ebc * pa[ea] * pac[eac] * pb[eb] * pmbc[ebc - 1];
            }
            U[p * n + q] = norm * u;
            if (Ua) Ua[p * n + q] = norm * ua;
            if (Uac) Uac[p * n + q] = norm * uac;
            if (Ub) Ub[p * n + q] = norm * ub;
            if (Ubc) Ubc[p * n + q] = norm * ubc;
        }
    }
}

void or_wigner_u(int tj, double are, double aim, double bre, double bim, double* out) {
    int n = tj + 1;
    cplx* U = (cplx*)malloc(sizeof(cplx) * n * n);
    wigner_u_partials(tj, are + I * aim, bre + I * bim, U, NULL, NULL, NULL, NULL);
    for (int e = 0; e < n * n; ++e) {
        out[2 * e] = creal(U[e]);
        out[2 * e + 1] = cimag(U[e]);
    }
    free(U);
}

int or_snap_triples(int twojmax, int* out) {
    int cnt = 0;
    for (int tj1 = 0; tj1 <= twojmax; ++tj1)
        for (int tj2 = 0; tj2 <= tj1; ++tj2)
            for (int tj = tj1; tj <= twojmax; ++tj) {
                if (tj > tj1 + tj2) continue;
                if ((tj1 + tj2 + tj) & 1) continue;
                if (out) {
                    out[3 * cnt] = tj1;
                    out[3 * cnt + 1] = tj2;
                    out[3 * cnt + 2] = tj;
                }
                ++cnt;
            }
    return cnt;
}

static void min_image(const double box[3], double d[3]) {
    for (int a = 0; a < 3; ++a) d[a] -= box[a] * nearbyint(d[a] / box[a]);
}

int or_neighbors(int natoms, const double* pos, const double box[3], double rc, int nmax, int* cnt,
                 int* list) {
    int maxc = 0, overflow = 0;
    for (int i = 0; i < natoms; ++i) {
        int c = 0;
        for (int k = 0; k < natoms; ++k) {
            if (k == i) continue;
            double d[3] = {pos[k] - pos[i], pos[natoms + k] - pos[natoms + i],
                           pos[2 * natoms + k] - pos[2 * natoms + i]};
            min_image(box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rc * rc) {
                if (c < nmax) list[i * nmax + c] = k;
                else overflow = 1;
                ++c;
            }
        }
        cnt[i] = c;
        if (c > maxc) maxc = c;
    }
    return overflow ? -1 : maxc;
}

/* per-call cache of CG values for every bispectrum triple */
typedef struct {
    int nt;
    int* tri;          /* [nt][3] */
    double** cgt;      /* per triple: [(tm1+tj1)/2][(tm2+tj2)/2] -> <j1 m1 j2 m2 | j m1+m2> */
    int uoff[32];      /* offset of level tj in the concatenated U arrays */
    int utot;          /* total number of U elements, sum (tj+1)^2 */
} snap_tables;

static void snap_tables_build(int twojmax, snap_tables* T) {
    T->nt = or_snap_triples(twojmax, NULL);
    T->tri = (int*)malloc(sizeof(int) * 3 * T->nt);
    or_snap_triples(twojmax, T->tri);
    T->cgt = (double**)malloc(sizeof(double*) * T->nt);
    for (int t = 0; t < T->nt; ++t) {
        int tj1 = T->tri[3 * t], tj2 = T->tri[3 * t + 1], tj = T->tri[3 * t + 2];
        double* c = (double*)malloc(sizeof(double) * (tj1 + 1) * (tj2 + 1));
        for (int p1 = 0; p1 <= tj1; ++p1)
            for (int p2 = 0; p2 <= tj2; ++p2) {
                int tm1 = 2 * p1 - tj1, tm2 = 2 * p2 - tj2;
                c[p1 * (tj2 + 1) + p2] = or_cg(tj1, tm1, tj2, tm2, tj, tm1 + tm2);
            }
        T->cgt[t] = c;
    }
    int off = 0;
    for (int tj = 0; tj <= twojmax; ++tj) {
        T->uoff[tj] = off;
        off += (tj + 1) * (tj + 1);
    }
    T->utot = off;
}

static void snap_tables_free(snap_tables* T) {
    for (int t = 0; t < T->nt; ++t) free(T->cgt[t]);
    free(T->cgt);
    free(T->tri);
}

/* One atom: energy E_i, bispectrum B_i[nt], and the gradients g[k][3] = dE_i/d r_ik for
   each neighbour (r_ik = r_k - r_i).  nb neighbour vectors rv[k][3]. */
static void snap_atom(const or_snap_params* p, const snap_tables* T, const double* beta, int nb,
                      const double* rv, double* Ei, double* Bi, double* g) {
    const int tJ = p->twojmax;
    const double kappa = p->rfac0 * M_PI / p->rcut;
    cplx* Utot = (cplx*)calloc(T->utot, sizeof(cplx));
    cplx* G = (cplx*)calloc(T->utot, sizeof(cplx));
    cplx* Uk = (cplx*)malloc(sizeof(cplx) * T->utot);
    cplx* Ua = (cplx*)malloc(sizeof(cplx) * T->utot);
    cplx* Uac = (cplx*)malloc(sizeof(cplx) * T->utot);
    cplx* Ub = (cplx*)malloc(sizeof(cplx) * T->utot);
    cplx* Ubc = (cplx*)malloc(sizeof(cplx) * T->utot);

    /* self term: w_self = 1 at g = identity, U^j(I) = I */
    for (int tj = 0; tj <= tJ; ++tj)
        for (int pp = 0; pp <= tj; ++pp) Utot[T->uoff[tj] + pp * (tj + 1) + pp] = 1.0;

    for (int k = 0; k < nb; ++k) {
        double x = rv[3 * k], y = rv[3 * k + 1], z = rv[3 * k + 2];
        double r = sqrt(x * x + y * y + z * z);
        double th = kappa * r;
        cplx a = cos(th) - I * sin(th) * z / r;
        cplx b = sin(th) * (y - I * x) / r;
        double w = p->switchflag ? 0.5 * (cos(M_PI * r / p->rcut) + 1.0) : 1.0;
        for (int tj = 0; tj <= tJ; ++tj) {
            wigner_u_partials(tj, a, b, Uk + T->uoff[tj], NULL, NULL, NULL, NULL);
            for (int e = 0; e < (tj + 1) * (tj + 1); ++e) Utot[T->uoff[tj] + e] += w * Uk[T->uoff[tj] + e];
        }
    }

    /* bispectrum and gradient G with dE_i = Re sum conj(G) dU_tot, by the product rule
       over the three factors of every triple (no symmetry identities used) */
    double E = beta[0];
    for (int t = 0; t < T->nt; ++t) {
        int tj1 = T->tri[3 * t], tj2 = T->tri[3 * t + 1], tj = T->tri[3 * t + 2];
        const double* c = T->cgt[t];
        const cplx* U1 = Utot + T->uoff[tj1];
        const cplx* U2 = Utot + T->uoff[tj2];
        const cplx* Uj = Utot + T->uoff[tj];
        cplx* G1 = G + T->uoff[tj1];
        cplx* G2 = G + T->uoff[tj2];
        cplx* Gj = G + T->uoff[tj];
        double bt = beta[1 + t];
        double Bsum = 0.0;
        for (int tm = -tj; tm <= tj; tm += 2)
            for (int tmp = -tj; tmp <= tj; tmp += 2) {
                cplx uj = Uj[((tm + tj) / 2) * (tj + 1) + (tmp + tj) / 2];
                for (int tm1 = -tj1; tm1 <= tj1; tm1 += 2) {
                    int tm2 = tm - tm1;
                    if (tm2 < -tj2 || tm2 > tj2) continue;
                    double c1 = c[((tm1 + tj1) / 2) * (tj2 + 1) + (tm2 + tj2) / 2];
                    for (int tm1p = -tj1; tm1p <= tj1; tm1p += 2) {
                        int tm2p = tmp - tm1p;
                        if (tm2p < -tj2 || tm2p > tj2) continue;
                        double c2 = c[((tm1p + tj1) / 2) * (tj2 + 1) + (tm2p + tj2) / 2];
                        double cc = c1 * c2;
                        if (cc == 0.0) continue;
                        int e1 = ((tm1 + tj1) / 2) * (tj1 + 1) + (tm1p + tj1) / 2;
                        int e2 = ((tm2 + tj2) / 2) * (tj2 + 1) + (tm2p + tj2) / 2;
                        int ej = ((tm + tj) / 2) * (tj + 1) + (tmp + tj) / 2;
                        cplx x12 = U1[e1] * U2[e2];
                        Bsum += creal(cc * conj(uj) * x12);
                        Gj[ej] += bt * cc * x12;
                        G1[e1] += bt * cc * uj * conj(U2[e2]);
                        G2[e2] += bt * cc * uj * conj(U1[e1]);
                    }
                }
            }
        if (Bi) Bi[t] = Bsum;
        E += bt * Bsum;
    }
    *Ei = E;

    /* chain rule through U(a(r), b(r)) and fc(r) for every neighbour */
    for (int k = 0; k < nb && g; ++k) {
        double x = rv[3 * k], y = rv[3 * k + 1], z = rv[3 * k + 2];
        double xyz[3] = {x, y, z};
        double r = sqrt(x * x + y * y + z * z);
        double th = kappa * r;
        double S = sin(th) / r;                                  /* sin(theta0)/r */
        double dS = (kappa * cos(th) * r - sin(th)) / (r * r);   /* dS/dr */
        cplx a = cos(th) - I * z * S;
        cplx b = (y - I * x) * S;
        double w = p->switchflag ? 0.5 * (cos(M_PI * r / p->rcut) + 1.0) : 1.0;
        double dw = p->switchflag ? -0.5 * sin(M_PI * r / p->rcut) * M_PI / p->rcut : 0.0;
        cplx da[3], db[3];
        for (int al = 0; al < 3; ++al) {
            double drdx = xyz[al] / r;
            da[al] = -kappa * sin(th) * drdx - I * ((al == 2 ? S : 0.0) + z * dS * drdx);
            db[al] = ((al == 1 ? 1.0 : 0.0) - I * (al == 0 ? 1.0 : 0.0)) * S + (y - I * x) * dS * drdx;
        }
        double gk[3] = {0, 0, 0};
        for (int tj = 0; tj <= tJ; ++tj) {
            int o = T->uoff[tj];
            wigner_u_partials(tj, a, b, Uk + o, Ua + o, Uac + o, Ub + o, Ubc + o);
            for (int e = 0; e < (tj + 1) * (tj + 1); ++e) {
                for (int al = 0; al < 3; ++al) {
                    double drdx = xyz[al] / r;
                    cplx dU = Ua[o + e] * da[al] + Uac[o + e] * conj(da[al]) + Ub[o + e] * db[al] +
                              Ubc[o + e] * conj(db[al]);
                    cplx dUtot = dw * drdx * Uk[o + e] + w * dU;
                    gk[al] += creal(conj(G[o + e]) * dUtot);
                }
            }
        }
        g[3 * k] = gk[0];
        g[3 * k + 1] = gk[1];
        g[3 * k + 2] = gk[2];
    }
    free(Utot); free(G); free(Uk); free(Ua); free(Uac); free(Ub); free(Ubc);
}

int or_snap_energy_forces(const or_snap_params* p, int nbatch, int natoms, const double box[3],
                          const double* pos, const double* beta, double* energy, double* forces,
                          double* sumB, double* Bat) {
    if (!p || p->twojmax < 0 || p->twojmax > 14 || p->rmin0 != 0.0 || natoms < 1 || nbatch < 0)
        return -1;
    snap_tables T;
    snap_tables_build(p->twojmax, &T);
    const int nt = T.nt;
    long nall = (long)nbatch * natoms;
    double* Ei = (double*)malloc(sizeof(double) * (nall > 0 ? nall : 1));
    double* Ball = (double*)malloc(sizeof(double) * (nall > 0 ? nall : 1) * nt);
    int* nnb = (int*)malloc(sizeof(int) * (nall > 0 ? nall : 1));
    int* nbidx = (int*)malloc(sizeof(int) * (nall > 0 ? nall : 1) * natoms);
    double* gall = (double*)malloc(sizeof(double) * (nall > 0 ? nall : 1) * natoms * 3);

#pragma omp parallel for schedule(dynamic) if (!omp_in_parallel())
    for (long ia = 0; ia < nall; ++ia) {
        int bb = (int)(ia / natoms), i = (int)(ia % natoms);
        const double* P = pos + (long)bb * 3 * natoms;
        double* rv = (double*)malloc(sizeof(double) * 3 * natoms);
        int nb = 0;
        for (int k = 0; k < natoms; ++k) {
            if (k == i) continue;
            double d[3] = {P[k] - P[i], P[natoms + k] - P[natoms + i], P[2 * natoms + k] - P[2 * natoms + i]};
            min_image(box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < p->rcut * p->rcut) {
                rv[3 * nb] = d[0]; rv[3 * nb + 1] = d[1]; rv[3 * nb + 2] = d[2];
                nbidx[ia * natoms + nb] = k;
                ++nb;
            }
        }
        nnb[ia] = nb;
        snap_atom(p, &T, beta, nb, rv, &Ei[ia], Ball + ia * nt, gall + ia * natoms * 3);
        free(rv);
    }

    for (int bb = 0; bb < nbatch; ++bb) {
        double E = 0.0;
        double* F = forces ? forces + (long)bb * 3 * natoms : NULL;
        if (F) memset(F, 0, sizeof(double) * 3 * natoms);
        for (int i = 0; i < natoms; ++i) {
            long ia = (long)bb * natoms + i;
            E += Ei[ia];
            for (int q = 0; q < nnb[ia] && F; ++q) {
                int k = nbidx[ia * natoms + q];
                for (int al = 0; al < 3; ++al) {
                    double gq = gall[(ia * natoms + q) * 3 + al];
                    F[al * natoms + k] -= gq;   /* -dE_i/dr_k */
                    F[al * natoms + i] += gq;   /* -dE_i/dr_i = +dE_i/dr_ik */
                }
            }
        }
        if (energy) energy[bb] = E;
        if (sumB) {
            double* sb = sumB + (long)bb * (1 + nt);
            sb[0] = (double)natoms;
            for (int t = 0; t < nt; ++t) {
                double s = 0.0;
                for (int i = 0; i < natoms; ++i) s += Ball[((long)bb * natoms + i) * nt + t];
                sb[1 + t] = s;
            }
        }
        if (Bat) memcpy(Bat + (long)bb * natoms * nt, Ball + (long)bb * natoms * nt, sizeof(double) * natoms * nt);
    }
    free(Ei); free(Ball); free(nnb); free(nbidx); free(gall);
    snap_tables_free(&T);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Finnis-Sinclair EAM (the coarse potential V_C, Sec. 3.1):
 *   rho_i = sum_{j != i, r_ij < d} (r_ij - d)^2
 *   E = sum_i -A sqrt(rho_i) + 1/2 sum_{i != j, r_ij < c} (r_ij - c)^2 (c0 + c1 r_ij + c2 r_ij^2)
 * Forces by the chain rule; F'(rho) = -A / (2 sqrt rho), taken as 0 when rho = 0.
 * ---------------------------------------------------------------------------------- */
int or_fs_energy_forces(const or_fs_params* p, int nbatch, int natoms, const double box[3],
                        const double* pos, double* energy, double* forces) {
    if (!p || natoms < 1 || nbatch < 0) return -1;
#pragma omp parallel for schedule(dynamic) if (!omp_in_parallel())
    for (int bb = 0; bb < nbatch; ++bb) {
        const double* P = pos + (long)bb * 3 * natoms;
        double* rho = (double*)calloc(natoms, sizeof(double));
        double* dF = (double*)calloc(natoms, sizeof(double));
        double E = 0.0;
        for (int i = 0; i < natoms; ++i)
            for (int j = 0; j < natoms; ++j) {
                if (j == i) continue;
                double d[3] = {P[j] - P[i], P[natoms + j] - P[natoms + i], P[2 * natoms + j] - P[2 * natoms + i]};
                min_image(box, d);
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (r < p->d) rho[i] += (r - p->d) * (r - p->d);
                if (r < p->c) E += 0.5 * (r - p->c) * (r - p->c) * (p->c0 + p->c1 * r + p->c2 * r * r);
            }
        for (int i = 0; i < natoms; ++i) {
            E += -p->A * sqrt(rho[i]);
            dF[i] = rho[i] > 0.0 ? -p->A / (2.0 * sqrt(rho[i])) : 0.0;
        }
        if (forces) {
            double* F = forces + (long)bb * 3 * natoms;
            memset(F, 0, sizeof(double) * 3 * natoms);
            for (int i = 0; i < natoms; ++i)
                for (int j = 0; j < natoms; ++j) {
                    if (j == i) continue;
                    double d[3] = {P[j] - P[i], P[natoms + j] - P[natoms + i], P[2 * natoms + j] - P[2 * natoms + i]};
                    min_image(box, d);
                    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    double dEdr = 0.0;
                    if (r < p->d) dEdr += (dF[i] + dF[j]) * 2.0 * (r - p->d);
                    if (r < p->c)
                        dEdr += 2.0 * (r - p->c) * (p->c0 + p->c1 * r + p->c2 * r * r) +
                                (r - p->c) * (r - p->c) * (p->c1 + 2.0 * p->c2 * r);
                    for (int al = 0; al < 3; ++al) F[al * natoms + i] += dEdr * d[al] / r;
                }
        }
        if (energy) energy[bb] = E;
        free(rho);
        free(dF);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Langevin propagation of one interval (Sec. 2, eqs. (2)-(3); corrected eqs. (11)-(12)).
 * With masses: the scheme acts on velocities v = p/m with force F/m and temperature
 * k_B T C_l / m (C_l the schedule of eqs. (13)-(14)):
 *   v_{l+1/2} = v_l + dt/2 a(q_l) - dt/2 gamma v_{l-1/2} + 1/2 sqrt(2 gamma kT C_l/m dt) G_l
 *   q_{l+1}   = q_l + dt v_{l+1/2}
 *   v_{l+1}   = v_{l+1/2} + dt/2 a(q_{l+1}) - dt/2 gamma v_{l+1/2} + 1/2 sqrt(2 gamma kT C_{l+1}/m dt) G_{l+1}
 * with v_{-1/2} := v_0 (the first iterate, eq. (2)).  Every call restarts at l = 0, as
 * LAMMPS does for each parareal interval (Sec. 2.3-2.4).
 * Option BAOAB (Leimkuhler-Matthews): B (half kick), A (half drift), O (exact OU step
 * with exp(-gamma dt)), A, B; one Gaussian G_l per step with the same keying.
 * ---------------------------------------------------------------------------------- */
static int forces_one(const or_potential* pot, int natoms, const double box[3], const double* q,
                      double* F) {
    if (pot->kind == OR_POT_SNAP)
        return or_snap_energy_forces(&pot->snap, 1, natoms, box, q, pot->beta, NULL, F, NULL, NULL);
    if (pot->kind == OR_POT_FS) return or_fs_energy_forces(&pot->fs, 1, natoms, box, q, NULL, F);
    if (pot->kind == OR_POT_ZERO) {
        memset(F, 0, sizeof(double) * 3 * natoms);
        return 0;
    }
    return -1;
}

static double schedule_C(int schedule, int ell) {
    if (schedule == OR_SCHED_ROBUST) return ell == 0 ? 3.0 : 1.0;   /* eq. (13) */
    if (schedule == OR_SCHED_L1_SYM) return 2.0;                    /* eq. (14), L = 1 only */
    return 1.0;
}

static int propagate_one(const or_potential* pot, int natoms, const double box[3], double* q,
                         double* v, int L, int64_t n, const or_langevin* lp) {
    const double dt = lp->dt, gam = lp->gamma;
    const double kT_m = OR_KB * lp->T / lp->mass * OR_FTOA;   /* Angstrom^2/ps^2 */
    const double f2a = OR_FTOA / lp->mass;                    /* eV/Angstrom -> Angstrom/ps^2 */
    double* F = (double*)malloc(sizeof(double) * 3 * natoms);
    double* vh = (double*)malloc(sizeof(double) * 3 * natoms);
    int rc = forces_one(pot, natoms, box, q, F);
    if (lp->scheme == OR_SCHEME_PAPER) {
        memcpy(vh, v, sizeof(double) * 3 * natoms);   /* v_{-1/2} := v_0 */
        for (int ell = 0; ell < L && rc == 0; ++ell) {
            double s0 = 0.5 * sqrt(2.0 * gam * kT_m * schedule_C(lp->schedule, ell) * dt);
            double s1 = 0.5 * sqrt(2.0 * gam * kT_m * schedule_C(lp->schedule, ell + 1) * dt);
            for (int i = 0; i < natoms; ++i) {
                double G[3];
                or_normals3(lp->seed, n, ell, i, G);
                for (int al = 0; al < 3; ++al) {
                    int e = al * natoms + i;
                    double vhalf = v[e] + 0.5 * dt * f2a * F[e] - 0.5 * dt * gam * vh[e] + s0 * G[al];
                    vh[e] = vhalf;
                    q[e] = q[e] + dt * vhalf;
                }
            }
            rc = forces_one(pot, natoms, box, q, F);
            for (int i = 0; i < natoms; ++i) {
                double G[3];
                or_normals3(lp->seed, n, ell + 1, i, G);
                for (int al = 0; al < 3; ++al) {
                    int e = al * natoms + i;
                    v[e] = vh[e] + 0.5 * dt * f2a * F[e] - 0.5 * dt * gam * vh[e] + s1 * G[al];
                }
            }
        }
    } else if (lp->scheme == OR_SCHEME_BAOAB) {
        double c1 = exp(-gam * dt);
        double c2 = sqrt(kT_m * (1.0 - c1 * c1));
        for (int ell = 0; ell < L && rc == 0; ++ell) {
            for (int i = 0; i < natoms; ++i) {
                double G[3];
                or_normals3(lp->seed, n, ell, i, G);
                for (int al = 0; al < 3; ++al) {
                    int e = al * natoms + i;
                    v[e] += 0.5 * dt * f2a * F[e];
                    q[e] += 0.5 * dt * v[e];
                    v[e] = c1 * v[e] + c2 * G[al];
                    q[e] += 0.5 * dt * v[e];
                }
            }
            rc = forces_one(pot, natoms, box, q, F);
            for (int e = 0; e < 3 * natoms; ++e) v[e] += 0.5 * dt * f2a * F[e];
        }
    } else {
        rc = -1;
    }
    free(F);
    free(vh);
    return rc;
}

int or_propagate(const or_potential* pot, int nbatch, int natoms, const double box[3], double* q,
                 double* v, const int32_t* nsteps, const int64_t* interval_id, const or_langevin* lp) {
    if (!pot || !lp || natoms < 1 || nbatch < 0) return -1;
    for (int bb = 0; bb < nbatch; ++bb) {
        if (nsteps[bb] < 0) return -1;
        if (lp->schedule == OR_SCHED_L1_SYM && nsteps[bb] > 1) return -1;
    }
    int bad = 0;
    /* members are independent; when there are many, run them in parallel (each force
       evaluation then runs on one thread), otherwise parallelise inside the force call */
    if (nbatch >= or_num_threads()) {
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
        for (int bb = 0; bb < nbatch; ++bb)
            bad |= propagate_one(pot, natoms, box, q + (long)bb * 3 * natoms, v + (long)bb * 3 * natoms,
                                 nsteps[bb], interval_id[bb], lp) != 0;
    } else {
        for (int bb = 0; bb < nbatch; ++bb)
            bad |= propagate_one(pot, natoms, box, q + (long)bb * 3 * natoms, v + (long)bb * 3 * natoms,
                                 nsteps[bb], interval_id[bb], lp) != 0;
    }
    return bad ? -1 : 0;
}
