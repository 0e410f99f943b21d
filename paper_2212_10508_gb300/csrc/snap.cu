// SNAP: host-side tables (Clebsch-Gordan blocks, contraction schedule) and the kernels behind
// snap_energy_forces (Sec. 3.1, fine potential).
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>

#include "pmd_internal.h"
#include "snap_kernels.cuh"

namespace pmd {

// ---- Clebsch-Gordan <j1 m1 j2 m2 | J M> (doubled arguments), Racah's closed form ---------
static double lfact(int n) { return std::lgamma((double)n + 1.0); }

static double clebsch(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
    if (tm1 + tm2 != tM || std::abs(tm1) > tj1 || std::abs(tm2) > tj2 || std::abs(tM) > tJ) return 0.0;
    if (tJ < std::abs(tj1 - tj2) || tJ > tj1 + tj2 || ((tj1 + tj2 + tJ) & 1)) return 0.0;
    const int a = (tj1 + tj2 - tJ) / 2, b = (tj1 - tm1) / 2, c = (tj2 + tm2) / 2;
    const int d = (tJ - tj2 + tm1) / 2, e = (tJ - tj1 - tm2) / 2;
    const double lpre = 0.5 * (std::log((double)tJ + 1.0) + lfact((tJ + tj1 - tj2) / 2) + lfact((tJ - tj1 + tj2) / 2) +
                               lfact(a) - lfact((tj1 + tj2 + tJ) / 2 + 1) + lfact((tj1 + tm1) / 2) + lfact(b) +
                               lfact((tj2 - tm2) / 2) + lfact(c) + lfact((tJ + tM) / 2) + lfact((tJ - tM) / 2));
    double s = 0.0;
    const int zlo = std::max(0, std::max(-d, -e)), zhi = std::min(a, std::min(b, c));
    for (int z = zlo; z <= zhi; ++z) {
        double t = std::exp(lpre - lfact(z) - lfact(a - z) - lfact(b - z) - lfact(c - z) - lfact(d + z) - lfact(e + z));
        s += (z & 1) ? -t : t;
    }
    return s;
}

// Jobs of the batched Y phase (lane = atom).  A job is one output row (tj, p) of the half
// layout of Y and one block (ta, tb, J = tj); it covers the row's h_ncol(tj) outputs.  The Y
// phase runs in stages of sub-block sizes (tb <= SB_SMALL_TB together, then one stage per larger
// tb) separated by CTA barriers, so that the CTA executes the unrolled code of few variants at a
// time.  A stage is a list of rows, longest first (cost model of the FP and load instructions);
// warps take rows from a shared counter, and a row's jobs of the stage run in a fixed order on the
// warp that took it.  Each output's update sequence is therefore fixed (stages in order, then the
// row's jobs in order) whatever warp runs it: the sums are deterministic.
// Rows i of U^a that a job visits, [ilo, ihi] (p1 = p + s - tb + i within 0..ta).  In a diagonal
// block (ta = tb) the rows i and i* = tb - p10 - i hold the same two factors swapped (p1 <-> p2, and
// every column pair likewise), with the same product of Clebsch-Gordan weights (their two sign
// factors (-1)^(a+b-J) cancel), so the two rows sum to the same value: the job visits i <= i* only
// and weights i < i* twice.
static void job_rows(int ta, int tb, int p10, int* ilo, int* ihi) {
    *ilo = p10 < 0 ? -p10 : 0;
    *ihi = std::min(tb, ta - p10);
    if (ta == tb) *ihi = std::min(*ihi, (tb - p10) / 2);
}

// First output column of a row job: rows p > J of an integer J skip the middle column q = J (m = 0),
// whose elements are mirror images of rows p < J: Y(p, J) = (-1)^(p-J) conj Y(2J - p, J).
static int job_first_col(int tj, int p) { return (tj % 2 == 0 && 2 * p > tj) ? 1 : 0; }

// Coefficient record of one job (float offset, a multiple of 4, into T->sb_coef): first the
// column weights c2[o][k] = <a q1, b tb-k | J q> with q = qlo + o0 + o, q1 = q + s - tb + k (zero
// where q1 is outside 0..ta), o < h_ncol(J) - o0, k <= tb; then the row weights c1[i] = <a p1, b tb-i | J p>
// with p1 = p + s - tb + i (zero outside 0..ta; doubled for the paired rows of a diagonal block);
// padded to a multiple of 4.
static int append_job_coefs(SnapHostTables* T, int blk, int tj, int p, int o0) {
    const int ta = T->blk_ta[blk], tb = T->blk_tb[blk], nc = ncol_half(tj) - o0;
    const double* cg = T->cg.data() + T->blk_cgoff[blk];
    const int s = (ta + tb - tj) / 2, p10 = p + s - tb, c0 = qlo(tj) + o0 + s - tb;
    const int off = (int)T->sb_coef.size();
    for (int o = 0; o < nc; ++o)
        for (int k = 0; k <= tb; ++k) {
            const int q1 = c0 + o + k;
            T->sb_coef.push_back(q1 >= 0 && q1 <= ta ? (float)cg[q1 * (tb + 1) + (tb - k)] : 0.f);
        }
    for (int i = 0; i <= tb; ++i) {
        const int p1 = p10 + i;
        const double w = (ta == tb && 2 * i < tb - p10) ? 2.0 : 1.0;
        T->sb_coef.push_back(p1 >= 0 && p1 <= ta ? (float)(w * cg[p1 * (tb + 1) + (tb - i)]) : 0.f);
    }
    while (T->sb_coef.size() % 4) T->sb_coef.push_back(0.f);
    return off;
}

static void build_batch_jobs(SnapHostTables* T) {
    struct RJ {
        int tj, p, blk, ta, tb;
    };
    const int nblk = (int)T->blk_ta.size();
    const int nstage = sb_num_stages(T->twojmax);
    std::vector<std::map<std::pair<int, int>, std::pair<double, std::vector<RJ>>>> stage(nstage);
    for (int tj = 0; tj <= T->twojmax; ++tj) {
        for (int p = 0; p <= tj; ++p)
            for (int id = 0; id < nblk; ++id) {
                const int nc = ncol_half(tj) - job_first_col(tj, p);
                if (T->blk_tj[id] != tj) continue;
                const int ta = T->blk_ta[id], tb = T->blk_tb[id];
                const int s = (ta + tb - tj) / 2, p10 = p + s - tb;
                int ilo, ihi;
                job_rows(ta, tb, p10, &ilo, &ihi);
                const int ni = ihi - ilo + 1;
                if (ni <= 0) continue;
                const int terms = nc * (tb + 1), loads = 2 * tb + nc + 1;   // branch-free windows
                auto& row = stage[sb_stage_of(tb)][{tj, p}];
                row.first += ni * (6.0 * terms + 2.0 * loads) + nc * (tb + 1) + 4.0 * nc + 20.0;
                row.second.push_back({tj, p, id, ta, tb});
            }
    }
    T->sb_jobs.clear();
    T->sb_rows.clear();
    T->sb_coef.clear();
    T->sb_sptr.assign(nstage + 1, 0);
    T->sb_groups.clear();
    T->sb_gptr.assign(2 * nstage * 2, 0);
    T->sb_load_max = 0.0;
    T->sb_load_avg = 0.0;
    for (int st = 0; st < nstage; ++st) {
        // rows by decreasing width (outputs per row), then decreasing cost: the costly rows first, and
        // rows of equal width adjacent (groups of 2 or 4 rows for multi-row warps)
        std::vector<std::pair<double, std::pair<int, int>>> rows;
        for (auto& kv : stage[st]) rows.push_back({kv.second.first, kv.first});
        auto width = [](const std::pair<int, int>& r) { return ncol_half(r.first) - job_first_col(r.first, r.second); };
        std::stable_sort(rows.begin(), rows.end(), [&](const auto& x, const auto& y) {
            const int wx = width(x.second), wy = width(y.second);
            return wx != wy ? wx > wy : x.first > y.first;
        });
        const int row0 = (int)T->sb_rows.size() / 2;
        // expected makespan of the greedy take-next order (for the record)
        std::vector<double> load(SB_WARPS, 0.0);
        for (auto& r : rows) {
            auto it = std::min_element(load.begin(), load.end());
            *it += r.first;
            std::vector<RJ> js = stage[st][r.second].second;
            std::stable_sort(js.begin(), js.end(), [](const RJ& x, const RJ& y) { return x.tb < y.tb; });
            const int j0 = (int)T->sb_jobs.size() / 4;
            for (const RJ& j : js) {
                int ilo, ihi;
                job_rows(j.ta, j.tb, j.p + (j.ta + j.tb - j.tj) / 2 - j.tb, &ilo, &ihi);
                const int o0 = job_first_col(j.tj, j.p);
                T->sb_jobs.push_back(j.ta | (j.tb << 4) | (j.tj << 8) | (j.p << 12) | (ilo << 16) | (ihi << 20) |
                                     (o0 << 24));
                T->sb_jobs.push_back(append_job_coefs(T, j.blk, j.tj, j.p, o0));
                T->sb_jobs.push_back(uoff_full(j.ta) | (uoff_full(j.tb) << 16));
                T->sb_jobs.push_back((T->hoff[j.tj] + j.p * ncol_half(j.tj) + o0) | (j.blk << 16));
            }
            T->sb_rows.push_back(j0);
            T->sb_rows.push_back((int)T->sb_jobs.size() / 4);
        }
        T->sb_sptr[st + 1] = (int)T->sb_rows.size() / 2;
        // row groups for multi-row warps (R = 2 and 4 rows of equal width per warp pass)
        for (int g = 0; g < 2; ++g) {
            const int R = g == 0 ? 2 : 4;
            T->sb_gptr[(g * nstage + st) * 2] = (int)T->sb_groups.size() / 2;
            for (size_t r = 0; r < rows.size();) {
                size_t e = r + 1;
                while (e < rows.size() && (int)(e - r) < R && width(rows[e].second) == width(rows[r].second)) ++e;
                T->sb_groups.push_back(row0 + (int)r);
                T->sb_groups.push_back((int)(e - r));
                r = e;
            }
            T->sb_gptr[(g * nstage + st) * 2 + 1] = (int)T->sb_groups.size() / 2;
        }
        double tot = 0.0;
        for (double x : load) tot += x;
        T->sb_load_max += *std::max_element(load.begin(), load.end());
        T->sb_load_avg += tot / SB_WARPS;
    }
}

int build_snap_tables(int twojmax, SnapHostTables* T) {
    T->twojmax = twojmax;
    T->tri.clear();
    for (int tj1 = 0; tj1 <= twojmax; ++tj1)
        for (int tj2 = 0; tj2 <= tj1; ++tj2)
            for (int tj = tj1; tj <= twojmax; ++tj)
                if (tj <= tj1 + tj2 && ((tj1 + tj2 + tj) & 1) == 0) {
                    T->tri.push_back(tj1);
                    T->tri.push_back(tj2);
                    T->tri.push_back(tj);
                }
    T->nB = (int)T->tri.size() / 3;
    T->hoff.assign(twojmax + 2, 0);
    for (int tj = 0; tj <= twojmax; ++tj) T->hoff[tj + 1] = T->hoff[tj] + (tj + 1) * ncol_half(tj);
    T->nhalf = T->hoff[twojmax + 1];
    T->nfull = uoff_full(twojmax + 1);

    // contraction blocks: dB_t = Re<Z^j_{j1j2}, dU^j> + (2j+1)/(2j1+1) Re<Z^{j1}_{j j2}, dU^{j1}>
    //                            + (2j+1)/(2j2+1) Re<Z^{j2}_{j j1}, dU^{j2}>
    std::map<std::tuple<int, int, int>, int> bid;   // (tj, ta, tb) -> block
    std::vector<std::vector<std::pair<int, double>>> contrib;
    auto add = [&](int tJ, int x, int y, int t, double coef) {
        const int ta = std::max(x, y), tb = std::min(x, y);
        auto key = std::make_tuple(tJ, ta, tb);
        auto it = bid.find(key);
        int id;
        if (it == bid.end()) {
            id = (int)contrib.size();
            bid[key] = id;
            contrib.emplace_back();
        } else {
            id = it->second;
        }
        contrib[id].push_back({t, coef});
        return id;
    };
    T->tri_blk.assign(T->nB, -1);
    for (int t = 0; t < T->nB; ++t) {
        const int tj1 = T->tri[3 * t], tj2 = T->tri[3 * t + 1], tj = T->tri[3 * t + 2];
        T->tri_blk[t] = add(tj, tj1, tj2, t, 1.0);
        add(tj1, tj, tj2, t, (tj + 1.0) / (tj1 + 1.0));
        add(tj2, tj, tj1, t, (tj + 1.0) / (tj2 + 1.0));
    }
    const int nblk = (int)contrib.size();
    T->blk_ta.assign(nblk, 0);
    T->blk_tb.assign(nblk, 0);
    T->blk_tj.assign(nblk, 0);
    T->blk_cgoff.assign(nblk, 0);
    T->cg.clear();
    for (auto& kv : bid) {
        const int id = kv.second;
        const int tJ = std::get<0>(kv.first), ta = std::get<1>(kv.first), tb = std::get<2>(kv.first);
        T->blk_tj[id] = tJ;
        T->blk_ta[id] = ta;
        T->blk_tb[id] = tb;
    }
    for (int id = 0; id < nblk; ++id) {
        const int ta = T->blk_ta[id], tb = T->blk_tb[id], tJ = T->blk_tj[id];
        T->blk_cgoff[id] = (int)T->cg.size();
        for (int p1 = 0; p1 <= ta; ++p1)
            for (int p2 = 0; p2 <= tb; ++p2) {
                const int tm1 = 2 * p1 - ta, tm2 = 2 * p2 - tb;
                T->cg.push_back(clebsch(ta, tm1, tb, tm2, tJ, tm1 + tm2));
            }
    }
    T->beff_ptr.assign(nblk + 1, 0);
    T->beff_t.clear();
    T->beff_c.clear();
    for (int id = 0; id < nblk; ++id) {
        for (auto& tc : contrib[id]) {
            T->beff_t.push_back(tc.first);
            T->beff_c.push_back(tc.second);
        }
        T->beff_ptr[id + 1] = (int)T->beff_t.size();
    }

    // Y jobs: every half element e = (tj, p, q) (row-major half index) receives one job per
    // block (ta, tb, J = tj); a job is a (tb+1) x (tb+1) loop over p1 = p+s-tb+i, q1 = q+s-tb+k.
    struct Job {
        int e, blk, tb, p10, q10, ta;
    };
    std::vector<std::vector<Job>> per_e(T->nhalf);
    T->total_terms = 0;
    for (int tj = 0; tj <= twojmax; ++tj)
        for (int p = 0; p <= tj; ++p)
            for (int q = qlo(tj); q <= tj; ++q) {
                const int e = T->hoff[tj] + p * ncol_half(tj) + (q - qlo(tj));
                for (int id = 0; id < nblk; ++id) {
                    if (T->blk_tj[id] != tj) continue;
                    const int ta = T->blk_ta[id], tb = T->blk_tb[id];
                    const int s = (ta + tb - tj) / 2;
                    const int np1 = std::min(ta, p + s) - std::max(0, p + s - tb) + 1;
                    const int nq1 = std::min(ta, q + s) - std::max(0, q + s - tb) + 1;
                    if (np1 <= 0 || nq1 <= 0) continue;
                    per_e[e].push_back({e, id, tb, p + s - tb, q + s - tb, ta});
                    T->total_terms += np1 * nq1;
                }
            }
    // assign whole outputs to lanes so that, per sub-block size tb, the largest per-lane job
    // count (the number of lockstep rounds of that size) stays small
    const int NTB = twojmax + 1;
    auto w2 = [](int tb) { return (double)(tb + 1) * (tb + 1); };
    std::vector<std::vector<int>> cnt(32, std::vector<int>(NTB, 0));
    std::vector<int> mx(NTB, 0);
    std::vector<double> load(32, 0.0);
    std::vector<int> order(T->nhalf);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> ecost(T->nhalf, 0.0);
    for (int e = 0; e < T->nhalf; ++e)
        for (const Job& j : per_e[e]) ecost[e] += w2(j.tb);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ecost[x] > ecost[y]; });
    std::vector<std::vector<int>> lane_out(32);
    for (int e : order) {
        std::vector<int> c(NTB, 0);
        for (const Job& j : per_e[e]) c[j.tb] += 1;
        int best = 0;
        double best_inc = 1e300, best_load = 1e300;
        for (int l = 0; l < 32; ++l) {
            double inc = 0.0;
            for (int tb = 0; tb < NTB; ++tb)
                if (c[tb]) inc += w2(tb) * std::max(0, cnt[l][tb] + c[tb] - mx[tb]);
            if (inc < best_inc || (inc == best_inc && load[l] < best_load)) {
                best = l;
                best_inc = inc;
                best_load = load[l];
            }
        }
        for (int tb = 0; tb < NTB; ++tb) {
            cnt[best][tb] += c[tb];
            mx[tb] = std::max(mx[tb], cnt[best][tb]);
        }
        load[best] += ecost[e];
        lane_out[best].push_back(e);
    }
    // rounds: for each tb, mx[tb] rounds; lane l runs its k-th job of that size in round k
    T->jobs.clear();
    T->round_tb.clear();
    T->padded_terms = 0;
    for (int tb = 0; tb < NTB; ++tb) {
        std::vector<std::vector<Job>> lj(32);
        for (int l = 0; l < 32; ++l) {
            std::sort(lane_out[l].begin(), lane_out[l].end());
            for (int e : lane_out[l])
                for (const Job& j : per_e[e])
                    if (j.tb == tb) lj[l].push_back(j);
        }
        for (int r = 0; r < mx[tb]; ++r) {
            T->round_tb.push_back((unsigned char)tb);
            T->padded_terms += 32.0 * w2(tb);
            for (int l = 0; l < 32; ++l) {
                if (r < (int)lj[l].size()) {
                    const Job& j = lj[l][r];
                    T->jobs.push_back(j.e | (j.blk << 16));
                    T->jobs.push_back((j.p10 + 32) | ((j.q10 + 32) << 8) | (j.ta << 16) | (tb << 24));
                    T->jobs.push_back(uoff_full(j.ta) | (uoff_full(tb) << 16));
                    T->jobs.push_back(T->blk_cgoff[j.blk]);
                } else {   // padding: every row/column out of range, output = the dummy slot
                    T->jobs.push_back(T->nhalf);
                    T->jobs.push_back(0 | (0 << 8) | (tb << 16) | (tb << 24));
                    T->jobs.push_back(0);
                    T->jobs.push_back(0);
                }
            }
        }
    }
    T->nrounds = (int)T->round_tb.size();
    build_batch_jobs(T);
    return PMD_OK;
}

template <typename real>
static int upload_tables(pmd_snap* s) {
    const SnapHostTables& T = s->T;
    int rc;
    std::vector<real> cg(T.cg.begin(), T.cg.end());
    if ((rc = s->d_cg.ensure(std::max<size_t>(1, cg.size()) * sizeof(real)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_cg.p, cg.data(), cg.size() * sizeof(real), cudaMemcpyHostToDevice));
    const int nblk = (int)T.blk_ta.size();
    std::vector<int4> blk(nblk);
    for (int i = 0; i < nblk; ++i) blk[i] = make_int4(T.blk_ta[i], T.blk_tb[i], T.blk_tj[i], T.blk_cgoff[i]);
    if ((rc = s->d_blk.ensure(nblk * sizeof(int4)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_blk.p, blk.data(), nblk * sizeof(int4), cudaMemcpyHostToDevice));
    if ((rc = s->d_beffptr.ensure((nblk + 1) * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_beffptr.p, T.beff_ptr.data(), (nblk + 1) * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_befft.ensure(T.beff_t.size() * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_befft.p, T.beff_t.data(), T.beff_t.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_beffc.ensure(T.beff_c.size() * sizeof(double)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_beffc.p, T.beff_c.data(), T.beff_c.size() * sizeof(double), cudaMemcpyHostToDevice));
    if ((rc = s->d_jobs.ensure(std::max<size_t>(1, T.jobs.size()) * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_jobs.p, T.jobs.data(), T.jobs.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_roundtb.ensure(std::max<size_t>(1, T.round_tb.size())))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_roundtb.p, T.round_tb.data(), T.round_tb.size(), cudaMemcpyHostToDevice));
    if ((rc = s->d_sbjobs.ensure(std::max<size_t>(1, T.sb_jobs.size()) * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_sbjobs.p, T.sb_jobs.data(), T.sb_jobs.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_sbcoef.ensure(std::max<size_t>(4, T.sb_coef.size()) * sizeof(float)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_sbcoef.p, T.sb_coef.data(), T.sb_coef.size() * sizeof(float), cudaMemcpyHostToDevice));
    if ((rc = s->d_sbrows.ensure(std::max<size_t>(1, T.sb_rows.size()) * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_sbrows.p, T.sb_rows.data(), T.sb_rows.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_sbgroups.ensure(std::max<size_t>(2, T.sb_groups.size()) * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_sbgroups.p, T.sb_groups.data(), T.sb_groups.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_sbgptr.ensure(T.sb_gptr.size() * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_sbgptr.p, T.sb_gptr.data(), T.sb_gptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = s->d_sbsptr.ensure(T.sb_sptr.size() * sizeof(int)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_sbsptr.p, T.sb_sptr.data(), T.sb_sptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<int4> tb(T.nB);
    for (int t = 0; t < T.nB; ++t) {
        const int b = T.tri_blk[t];
        tb[t] = make_int4(b, T.blk_ta[b], T.blk_tb[b], T.blk_tj[b]);
    }
    if ((rc = s->d_triblk.ensure(std::max(1, T.nB) * sizeof(int4)))) return rc;
    PMD_CUDA_TRY(cudaMemcpy(s->d_triblk.p, tb.data(), T.nB * sizeof(int4), cudaMemcpyHostToDevice));
    return PMD_OK;
}

int snap_upload(pmd_snap* s) {
    return s->p.precision == PMD_FP64 ? upload_tables<double>(s) : upload_tables<float>(s);
}

SnapView snap_view(const pmd_snap* s, const double* beta) {
    SnapView v;
    v.cg = s->d_cg.p;
    v.beffptr = s->d_beffptr.as<int>();
    v.befft = s->d_befft.as<int>();
    v.beffc = s->d_beffc.as<double>();
    v.yt.jobs = s->d_jobs.as<int4>();
    v.yt.round_tb = s->d_roundtb.as<unsigned char>();
    v.yt.nrounds = s->T.nrounds;
    v.sbjobs = s->d_sbjobs.as<int4>();
    v.sbrows = s->d_sbrows.as<int2>();
    v.sbcoef = s->d_sbcoef.as<float>();
    v.sbsptr = s->d_sbsptr.as<int>();
    v.sbgroups = s->d_sbgroups.as<int2>();
    v.sbgptr = s->d_sbgptr.as<int>();
    v.beta = beta;
    v.ncg = (int)s->T.cg.size();
    v.nblk = (int)s->T.blk_ta.size();
    v.nB = s->T.nB;
    v.sp.rcut = s->p.rcut;
    v.sp.rcut_f = (float)s->p.rcut;
    v.sp.rfac0 = s->p.rfac0;
    v.sp.switchflag = s->p.switchflag;
    return v;
}

}  // namespace pmd

#include "snap_launch.cuh"

namespace pmd {

int snap_launch_large(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                      double* energy, double* forces, double* sumB, const SnapScratch& sc, cudaStream_t st);

// bytes of each scratch array for na atoms (forces always; U_tot and B only for energies)
void snap_scratch_sizes(const pmd_snap* s, long na, bool want_B, size_t sz[6]) {
    const size_t rs = s->p.precision == PMD_FP64 ? 8 : 4;
    sz[0] = (size_t)na * NMAX * sizeof(int);                          // nbr
    sz[1] = (size_t)na * sizeof(int);                                 // nnb
    sz[2] = (size_t)na * NMAX * 3 * rs;                               // dedr
    sz[3] = (size_t)na * sizeof(float4);                              // qf
    sz[4] = want_B ? (size_t)na * (size_t)s->T.nfull * 2 * rs : 0;    // utot
    sz[5] = want_B ? (size_t)na * (size_t)std::max(1, s->T.nB) * sizeof(double) : 0;   // B
}

int snap_compute_scratch(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                         double* energy, double* forces, double* sumB, const SnapScratch& sc, cudaStream_t st) {
    const bool f64 = s->p.precision == PMD_FP64;
    auto big32 = [] { return fail(PMD_EUNSUPPORTED, "twojmax > 8 is available in FP64 only"); };
    switch (s->p.twojmax) {
#define PMD_SNAP_CASE(TJV)                                                                                    \
    case TJV:                                                                                                 \
        return f64 ? launch_snap<double, TJV>(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st)     \
                   : launch_snap<float, TJV>(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st);
        PMD_SNAP_CASE(2)
        PMD_SNAP_CASE(4)
        PMD_SNAP_CASE(6)
        PMD_SNAP_CASE(8)
#undef PMD_SNAP_CASE
        // larger band limits (2J = 14 is the paper's SNAP-205): FP64 only, warp per atom
        case 10:
        case 12:
        case 14:
            return f64 ? snap_launch_large(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st) : big32();
    }
    return fail(PMD_EUNSUPPORTED, "twojmax must be 2, 4, 6, 8, 10, 12 or 14");
}

int snap_reserve_impl(pmd_snap* s, long na) {
    const size_t rs = s->p.precision == PMD_FP64 ? 8 : 4;
    int rc;
    if ((rc = s->s_nbr.ensure(na * NMAX * sizeof(int)))) return rc;
    if ((rc = s->s_nnb.ensure(na * sizeof(int)))) return rc;
    if ((rc = s->s_dedr.ensure(na * NMAX * 3 * rs))) return rc;
    if ((rc = s->s_qf.ensure(na * sizeof(float4)))) return rc;
    if ((rc = s->s_utot.ensure(na * (size_t)s->T.nfull * 2 * rs))) return rc;
    if ((rc = s->s_B.ensure(na * (size_t)std::max(1, s->T.nB) * sizeof(double)))) return rc;
    return PMD_OK;
}

int snap_compute(pmd_snap* s, int nbatch, int n, const double box[3], const double* pos, const double* beta,
                 double* energy, double* forces, double* sumB, cudaStream_t st) {
    int rc = snap_reserve_impl(s, (long)nbatch * n);
    if (rc) return rc;
    SnapScratch sc{s->s_nbr.as<int>(), s->s_nnb.as<int>(), s->s_dedr.p, s->s_qf.as<float4>(), s->s_utot.p,
                   s->s_B.as<double>()};
    return snap_compute_scratch(s, nbatch, n, box, pos, beta, energy, forces, sumB, sc, st);
}

}  // namespace pmd
