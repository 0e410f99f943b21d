// adaptive_restart: Algorithm 2 of the paper (Sec. 2.2) as an event-driven host state machine,
// and the cost / gain model of eqs. (7)-(9).
//
// Algorithm 2, restated: a slab [N_init, N_final] starts with N_final = N after a coarse
// initialisation.  Each parareal iteration on it runs the fine batch and the correction
// sweep; the sweep returns the relative error delta and, if delta exceeded delta_expl at
// interval n, n_stop = n.  Then:
//   delta > delta_expl : N_final := n_stop (shortened slab, same N_init) and iterate again;
//   delta < delta_conv : the slab is converged; the next slab is [N_final, N];
//   otherwise          : iterate again on the same slab.
// The run ends when a converged slab reaches N.  Reading for the degenerate case n_stop =
// N_init (Algorithm 2 would leave an empty slab): the slab becomes [N_init, N_init + 1],
// whose only interval is already exact after the iteration just run.
#include <cmath>
#include <vector>

#include "pmd_internal.h"

struct pmd_adaptive {
    int N = 0;
    double dconv = 0, dexpl = 0;
    int n_in = 0, n_fin = 0;
    int phase = 0;      // 0: not started, 1: iterating, 2: done
    int slab = -1;      // index of the current slab
    int k_slab = 0;     // iterations on the current slab
    struct Entry {
        int slab, n_in, n_fin, k;
    };
    std::vector<Entry> log;
};

extern "C" int pmd_adaptive_create(int N, double delta_conv, double delta_expl, pmd_adaptive** out) {
    if (!out) return pmd::fail(PMD_EINVAL, "pmd_adaptive_create: out is NULL");
    if (N < 0 || !(delta_conv > 0) || !(delta_expl > delta_conv))
        return pmd::fail(PMD_EINVAL, "pmd_adaptive_create: need N >= 0 and 0 < delta_conv < delta_expl");
    pmd_adaptive* st = new (std::nothrow) pmd_adaptive();
    if (!st) return pmd::fail(PMD_ENOMEM, "pmd_adaptive_create: out of host memory");
    st->N = N;
    st->dconv = delta_conv;
    st->dexpl = delta_expl;
    *out = st;
    return PMD_OK;
}

extern "C" int pmd_adaptive_destroy(pmd_adaptive* st) {
    delete st;
    return PMD_OK;
}

static void open_slab(pmd_adaptive* st, int n_in, pmd_action* next) {
    st->n_in = n_in;
    st->n_fin = st->N;
    st->slab += 1;
    st->k_slab = 0;
    st->log.push_back({st->slab, st->n_in, st->n_fin, 0});
    next->kind = PMD_ACT_ITERATE;
    next->n_in = st->n_in;
    next->n_fin = st->n_fin;
    next->open_slab = 1;
    next->k = 0;
}

static void done(pmd_adaptive* st, pmd_action* next) {
    st->phase = 2;
    next->kind = PMD_ACT_DONE;
    next->n_in = st->n_in;
    next->n_fin = st->n_fin;
    next->open_slab = 0;
    next->k = st->k_slab;
}

extern "C" int adaptive_restart(pmd_adaptive* st, double delta, int n_stop, pmd_action* next) {
    if (!st || !next) return pmd::fail(PMD_EINVAL, "adaptive_restart: NULL argument");
    if (st->phase == 2) {
        done(st, next);
        return PMD_OK;
    }
    if (st->phase == 0) {
        st->phase = 1;
        if (st->N == 0) {
            done(st, next);
            return PMD_OK;
        }
        open_slab(st, 0, next);
        return PMD_OK;
    }
    // report of the iteration just run on [n_in, n_fin]
    st->log.back().k += 1;
    st->k_slab += 1;
    if (std::isnan(delta) || delta > st->dexpl) {
        if (n_stop < st->n_in || n_stop > st->n_fin)
            return pmd::fail(PMD_EINVAL, "adaptive_restart: n_stop outside the current slab");
        int nf = n_stop > st->n_in ? n_stop : st->n_in + 1;
        st->n_fin = nf;
        if (st->n_fin >= st->N) {
            done(st, next);
            return PMD_OK;
        }
        st->log.push_back({st->slab, st->n_in, st->n_fin, 0});
        next->kind = PMD_ACT_ITERATE;
        next->n_in = st->n_in;
        next->n_fin = st->n_fin;
        next->open_slab = 0;
        next->k = st->k_slab;
        return PMD_OK;
    }
    if (delta < st->dconv) {
        if (st->n_fin >= st->N) {
            done(st, next);
            return PMD_OK;
        }
        open_slab(st, st->n_fin, next);
        return PMD_OK;
    }
    next->kind = PMD_ACT_ITERATE;
    next->n_in = st->n_in;
    next->n_fin = st->n_fin;
    next->open_slab = 0;
    next->k = st->k_slab;
    return PMD_OK;
}

extern "C" int pmd_adaptive_cost(const pmd_adaptive* st, double C_f, double C_c, double* cost, double* gamma_adapt,
                                 double* gamma_ideal) {
    if (!st) return pmd::fail(PMD_EINVAL, "pmd_adaptive_cost: NULL state");
    double c = 0.0;
    long ksum = 0;
    int last_slab = -1;
    for (const auto& e : st->log) {
        if (e.slab != last_slab) {
            c += (double)(st->N - e.n_in) * C_c;   // coarse initialisation of the slab
            last_slab = e.slab;
        }
        c += (double)e.k * ((C_f + C_c) + (double)(e.n_fin - e.n_in) * C_c);
        ksum += e.k;
    }
    if (cost) *cost = c;
    if (gamma_adapt) *gamma_adapt = c > 0 ? (double)st->N * C_f / c : 0.0;
    if (gamma_ideal) *gamma_ideal = ksum > 0 ? (double)st->N / (double)ksum : 0.0;
    return PMD_OK;
}

extern "C" int pmd_adaptive_log(const pmd_adaptive* st, int capacity, int* n_init, int* n_final, int* k, int* slab) {
    if (!st) return pmd::fail(PMD_EINVAL, "pmd_adaptive_log: NULL state");
    const int cnt = (int)st->log.size();
    for (int i = 0; i < cnt && i < capacity; ++i) {
        if (n_init) n_init[i] = st->log[i].n_in;
        if (n_final) n_final[i] = st->log[i].n_fin;
        if (k) k[i] = st->log[i].k;
        if (slab) slab[i] = st->log[i].slab;
    }
    return cnt;
}
