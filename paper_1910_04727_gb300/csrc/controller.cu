// The MLMC / MLQMC sample-size controller as a host routine over callbacks
// (Sec. 2.3, Sec. 2.4, Algorithms 1-3: the finest level fixed, or grown
// until the Richardson bias estimate passes).
//
// The controller owns no device state: the caller's `enqueue` adds samples
// of one (extended) level to its running sums, `read` returns them, and,
// with several ranks, `allgather` collects every rank's sums.  Each request
// [first, first + n) is split into contiguous per-rank shares
// (fm_shard_range), so rank r draws exactly the samples a single process
// would draw for those ids, and the sums of all ranks are folded in rank
// order: every rank sees the same totals and computes the same schedule,
// and the union of the ranks' samples is the single-process sample set.
// No CUDA call is made here.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fmgmlmc.h"

namespace {

constexpr double kMaxSamplesPerLevel = 1e9;   // guard against a runaway sample-size rule

void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// totals[cell] = fold over ranks (in rank order) of all[rank][cell]
void fold_ranks(const fm_level_sums* all, int world, size_t cells, fm_level_sums* totals) {
    for (size_t k = 0; k < cells; ++k) {
        fm_level_sums t;
        std::memset(&t, 0, sizeof(t));
        for (int r = 0; r < world; ++r) {
            const fm_level_sums& a = all[(size_t)r * cells + k];
            const double* src[4] = {a.sum_y, a.sum_y2, a.sum_qf, a.sum_qc};
            double* dst[4] = {t.sum_y, t.sum_y2, t.sum_qf, t.sum_qc};
            for (int q = 0; q < 4; ++q) {
                neumaier(dst[q][0], dst[q][1], src[q][0]);
                dst[q][1] += src[q][1];
            }
            t.count += a.count;
        }
        totals[k] = t;
    }
}

// Double-double helpers (Dekker 1971; Knuth's two-sum): a value is the
// unevaluated sum hi + lo.
struct DD {
    double hi, lo;
};

DD two_sum(double a, double b) {
    const double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

DD dd_add(DD a, DD b) {
    const DD s = two_sum(a.hi, b.hi);
    return two_sum(s.hi, s.lo + a.lo + b.lo);
}

DD dd_mul(DD a, DD b) {
    const double p = a.hi * b.hi;
    const double e = std::fma(a.hi, b.hi, -p);
    return two_sum(p, e + (a.hi * b.lo + a.lo * b.hi));
}

DD dd_div(DD a, double d) {
    const double q = a.hi / d;
    // remainder a - q d, formed exactly to first order
    const DD qd = dd_mul({q, 0.0}, {d, 0.0});
    const DD r = dd_add(a, {-qd.hi, -qd.lo});
    return two_sum(q, (r.hi + r.lo) / d);
}

// Mean and Bessel-corrected variance of one level-sum cell.  The sums are
// Neumaier pairs (sum, compensation) of Y and Y^2 (Y^2 accumulated with its
// exact rounding error), read as double-double numbers; S2 - S1^2 / n is
// formed in double-double, so the cancellation when |mean| >> sd costs
// nothing until sd / |mean| nears 1e-16.
void level_mean_var(const fm_level_sums& s, double* mean, double* var) {
    const double n = s.count;
    const DD s1 = two_sum(s.sum_y[0], s.sum_y[1]);
    const DD s2 = two_sum(s.sum_y2[0], s.sum_y2[1]);
    *mean = n > 0 ? (s1.hi + s1.lo) / n : NAN;
    if (!(n > 1)) {
        *var = 0.0;
        return;
    }
    const DD sq = dd_div(dd_mul(s1, s1), n);
    const DD d = dd_add(s2, {-sq.hi, -sq.lo});
    *var = std::max(0.0, (d.hi + d.lo) / (n - 1));
}

void set_err(char* err, size_t len, const std::string& msg) {
    if (err && len) std::snprintf(err, len, "%s", msg.c_str());
}

}  // namespace

extern "C" fm_status fm_level_stats(const fm_level_sums* sums, fm_level_stat* out) {
    if (!sums || !out) return FM_EINVAL;
    out->count = sums->count;
    level_mean_var(*sums, &out->mean, &out->var);
    out->sum_qf = sums->sum_qf[0] + sums->sum_qf[1];
    out->sum_qc = sums->sum_qc[0] + sums->sum_qc[1];
    return FM_OK;
}

extern "C" void fm_shard_range(uint64_t first, uint64_t n, int32_t rank, int32_t world, uint64_t* my_first,
                               uint64_t* my_n) {
    if (world < 1) world = 1;
    if (rank < 0 || rank >= world) {
        if (my_first) *my_first = first + n;
        if (my_n) *my_n = 0;
        return;
    }
    const uint64_t base = n / (uint64_t)world, extra = n % (uint64_t)world;
    const uint64_t r = (uint64_t)rank;
    const uint64_t count = base + (r < extra ? 1 : 0);
    const uint64_t start = first + r * base + std::min<uint64_t>(r, extra);
    if (my_first) *my_first = start;
    if (my_n) *my_n = count;
}

extern "C" fm_status mlmc_estimate_core(const fm_core_opts* o, fm_enqueue_fn enqueue, fm_read_fn read,
                                        fm_allgather_fn allgather, void* user, fm_core_result* out, char* err,
                                        size_t errlen) {
    if (!o || !enqueue || !read || !out) {
        set_err(err, errlen, "mlmc_estimate_core: null argument");
        return FM_EINVAL;
    }
    const int Emax = o->n_ext;
    const int R = o->qmc ? o->n_shifts : 1;
    const int world = o->world > 0 ? o->world : 1;
    const int lv0 = o->level0;
    if (Emax < 1 || Emax > FM_MAX_LEVELS + 1 || !o->cost || !(o->eps > 0) || o->n_pilot < 2 ||
        (o->qmc && (R < 2 || R > 64)) || o->rank < 0 || o->rank >= world || (world > 1 && !allgather) ||
        lv0 < 0 || lv0 >= Emax) {
        set_err(err, errlen, "mlmc_estimate_core: bad options (levels, cost, eps, n_pilot >= 2, shifts, rank)");
        return FM_EINVAL;
    }
    if (o->adapt && (o->n_ext_start < lv0 + 2 || o->n_ext_start > Emax)) {
        set_err(err, errlen, "mlmc_estimate_core: adapt needs level0 + 2 <= n_ext_start <= n_ext");
        return FM_EINVAL;
    }
    for (int e = 0; e < Emax; ++e)
        if (!(o->cost[e] > 0)) {
            set_err(err, errlen, "mlmc_estimate_core: costs must be positive");
            return FM_EINVAL;
        }
    const int max_rounds = o->max_rounds > 0 ? o->max_rounds : 100;
    const size_t cells = (size_t)Emax * R;
    std::vector<fm_level_sums> local(cells), all(cells * world), tot(cells);
    std::memset(out, 0, sizeof(*out));
    int64_t N[FM_MAX_LEVELS + 1] = {};
    double mean[FM_MAX_LEVELS + 1] = {}, var[FM_MAX_LEVELS + 1] = {};
    int E = o->adapt ? o->n_ext_start : Emax;   // extended levels in use

    // this rank's share of samples first .. first+n-1 of extended level e, every shift
    auto draw = [&](int e, int64_t first, int64_t n) -> fm_status {
        uint64_t f = 0, m = 0;
        fm_shard_range((uint64_t)first, (uint64_t)n, o->rank, world, &f, &m);
        if (m == 0) return FM_OK;
        for (int r = 0; r < R; ++r) {
            const fm_status st = enqueue(user, e, f, m, o->qmc ? r : -1);
            if (st != FM_OK) return st;
        }
        return FM_OK;
    };
    // every rank's sums, folded in rank order, then the statistics of the levels in use
    auto refresh = [&]() -> fm_status {
        fm_status st = read(user, local.data());
        if (st != FM_OK) return st;
        if (world > 1) {
            st = allgather(user, local.data(), all.data(), cells * sizeof(fm_level_sums));
            if (st != FM_OK) return st;
        } else {
            std::memcpy(all.data(), local.data(), cells * sizeof(fm_level_sums));
        }
        fold_ranks(all.data(), world, cells, tot.data());
        for (int e = 0; e < E; ++e) {
            if (!o->qmc) {
                const fm_level_sums& s = tot[e];
                const double n = s.count;
                const double sy = s.sum_y[0] + s.sum_y[1], sy2 = s.sum_y2[0] + s.sum_y2[1];
                if (!std::isfinite(sy) || !std::isfinite(sy2)) {
                    set_err(err, errlen, "mlmc_estimate: non-finite samples on level " + std::to_string(e));
                    return FM_ENOTCONV;
                }
                (void)n;
                level_mean_var(s, &mean[e], &var[e]);
            } else {
                double m[64];
                double mm = 0.0;
                for (int r = 0; r < R; ++r) {
                    const fm_level_sums& s = tot[(size_t)e * R + r];
                    m[r] = (s.sum_y[0] + s.sum_y[1]) / s.count;
                    if (!std::isfinite(m[r])) {
                        set_err(err, errlen, "mlmc_estimate: non-finite samples on level " + std::to_string(e));
                        return FM_ENOTCONV;
                    }
                    mm += m[r];
                }
                mm /= R;
                double v = 0.0;
                for (int r = 0; r < R; ++r) v += (m[r] - mm) * (m[r] - mm);
                mean[e] = mm;
                var[e] = v / ((double)R * (R - 1));
            }
        }
        return FM_OK;
    };
    // Richardson estimate of the weak error (Algorithm 1): |mean(Y_L)| /
    // (2^alpha - 1), alpha the caller's or the least-squares slope of
    // -log2|mean(Y_l)| over l = 1 .. L, floored at 1/2 so that a noisy fit of
    // a few levels cannot drive the denominator to 0.
    auto bias_estimate = [&](double* alpha_used) -> double {
        const int L = E - 1 - lv0;
        if (L < 1) {
            *alpha_used = NAN;
            return NAN;
        }
        double a = o->alpha;
        if (!(a > 0)) {
            double sx = 0, sy = 0, sxx = 0, sxy = 0;
            bool ok = L >= 2;
            for (int l = 1; l <= L && ok; ++l) {
                const double v = std::fabs(mean[lv0 + l]);
                if (!(v > 0)) ok = false;
                const double y = std::log2(v);
                sx += l;
                sy += y;
                sxx += (double)l * l;
                sxy += l * y;
            }
            const double n = L;
            const double fit = ok ? -(n * sxy - sx * sy) / (n * sxx - sx * sx) : NAN;
            a = std::isfinite(fit) ? std::max(fit, 0.5) : 0.5;
        }
        *alpha_used = a;
        return std::fabs(mean[E - 1]) / (std::pow(2.0, a) - 1.0);
    };
    const double bias_bar = o->eps / std::sqrt(2.0);

    int rounds = 0;
    if (!o->qmc) {
        // Algorithms 1 / 3: evaluate dN, update V_l and the optimal
        // N_l = ceil((2/eps^2) sqrt(V_l/C_l) sum_k sqrt(V_k C_k)), repeat; when
        // no level needs more samples, the bias test (adapt) adds a level.
        int64_t dN[FM_MAX_LEVELS + 1] = {};
        for (int e = 0; e < E; ++e) dN[e] = o->n_pilot;
        while (rounds < max_rounds) {
            bool any = false;
            for (int e = 0; e < E; ++e)
                if (dN[e] > 0) {
                    const fm_status st = draw(e, N[e], dN[e]);
                    if (st != FM_OK) return st;
                    N[e] += dN[e];
                    any = true;
                }
            if (!any) break;
            ++rounds;
            const fm_status st = refresh();
            if (st != FM_OK) return st;
            double tot_vc = 0.0;
            for (int e = 0; e < E; ++e) tot_vc += std::sqrt(var[e] * o->cost[e]);
            bool more = false;
            for (int e = 0; e < E; ++e) {
                const double opt = std::ceil(2.0 / (o->eps * o->eps) * std::sqrt(var[e] / o->cost[e]) * tot_vc);
                if (!std::isfinite(opt) || opt > kMaxSamplesPerLevel) {
                    set_err(err, errlen, "mlmc_estimate: level " + std::to_string(e) + " would need " +
                                             std::to_string(opt) + " samples (variance " + std::to_string(var[e]) +
                                             "); beyond the per-level cap");
                    return FM_ENOTCONV;
                }
                dN[e] = std::max<int64_t>(0, (int64_t)opt - N[e]);
                more = more || dN[e] > 0;
            }
            if (more || !o->adapt) continue;
            double a;
            if (bias_estimate(&a) < bias_bar || E == Emax) break;
            dN[E] = o->n_pilot;
            ++E;
        }
        double v = 0.0;
        for (int e = 0; e < E; ++e) v += var[e] / (double)N[e];
        out->var_estimator = v;
    } else {
        // Algorithm 2: pilot, then double N_l at argmax V[Y_l]/(N_l C_l) while
        // the variance is too large; then the bias test (adapt) adds a level.
        for (int e = 0; e < E; ++e) {
            const fm_status st = draw(e, 0, o->n_pilot);
            if (st != FM_OK) return st;
            N[e] = o->n_pilot;
        }
        fm_status st = refresh();
        if (st != FM_OK) return st;
        while (rounds < max_rounds) {
            double tot_v = 0.0;
            for (int e = 0; e < E; ++e) tot_v += var[e];
            if (tot_v <= o->eps * o->eps / 2) {
                double a;
                if (!o->adapt || bias_estimate(&a) < bias_bar || E == Emax) break;
                st = draw(E, 0, o->n_pilot);
                if (st != FM_OK) return st;
                N[E] = o->n_pilot;
                ++E;
            } else {
                int best = 0;
                double bv = -1.0;
                for (int e = 0; e < E; ++e) {
                    const double v = var[e] / ((double)N[e] * o->cost[e]);
                    if (v > bv) {
                        bv = v;
                        best = e;
                    }
                }
                if (N[best] > ((int64_t)1 << 31)) {
                    set_err(err, errlen, "mlmc_estimate: QMC point budget exhausted");
                    return FM_ENOTCONV;
                }
                st = draw(best, N[best], N[best]);
                if (st != FM_OK) return st;
                N[best] *= 2;
            }
            ++rounds;
            st = refresh();
            if (st != FM_OK) return st;
        }
        double v = 0.0;
        for (int e = 0; e < E; ++e) v += var[e];
        out->var_estimator = v;
    }
    double est = 0.0;
    for (int e = 0; e < E; ++e) {
        est += mean[e];
        out->mean[e] = mean[e];
        out->var[e] = var[e];
        out->N[e] = N[e];
    }
    out->estimate = est;
    out->rounds = rounds;
    out->n_ext_used = E;
    out->bias = bias_estimate(&out->alpha_used);
    out->bias_ok = out->bias < bias_bar ? 1 : 0;
    return FM_OK;
}
