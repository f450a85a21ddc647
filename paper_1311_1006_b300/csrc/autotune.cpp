// Autotuner: Algorithm 4 ("AT3b", Sec. 4.2) of the paper, a directed walk in
// N_levels whose moves that degrade the run time are re-tried only after
// enough accepted evaluations that the accumulated cost of the bad moves stays
// below a user cap on the relative tuning cost.  Noise is filtered as in
// Sec. 4.2.1: every decision compares the minimum time over a short window of
// evaluations.  Optionally theta is tuned too (the theta moves of Algorithms
// 2-4): theta moves alternate with N_levels moves, step 0.01 x fib(fibcount);
// a rejected theta move reverses direction and takes the next Fibonacci step,
// and at the end of the sequence the count restarts at 1 and the sequence
// grows by one (the growing step of Algorithm 2).  p follows theta through the
// tolerance: p = ceil(0.9 ln(TOL) / ln(theta)), the p ~ log TOL / log theta
// rule of Sec. 4.1 with the constant chosen so that p is never below Table 4.1
// (it equals the table or exceeds it by one at all 15 entries).  The
// load-balance variant AT3a has no counterpart: the whole evaluation runs on
// one device.
//
// Reading of the cost formulas (printed garbled in the paper):
//   upcost  += cost                                   (time lost by the rejected up-move)
//   uptime   = (upcost + cost)/cap - basetime         (base time still needed for the cap)
//   upinterval = uptime / (basetime / accepted evals) (evaluations to wait before moving up again)
// and the same for down-moves.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "fmm_internal.cuh"

using namespace fmm;


static double vmin(const std::vector<double>& v) { return *std::min_element(v.begin(), v.end()); }

namespace fmm {

static int fib(int n) {  // 1, 2, 3, 5, 8, ...
    int a = 1, b = 2;
    for (int i = 1; i < n; ++i) {
        const int c = a + b;
        a = b;
        b = c;
    }
    return a;
}

int p_for_tolerance(double tol, double theta) {
    if (!(tol > 0.0 && tol < 1.0) || !(theta > 0.0 && theta < 1.0)) return -1;
    const double q = 0.9 * std::log(tol) / std::log(theta);
    return std::max(1, (int)std::ceil(q - 1e-9));
}

// Largest theta of the range whose p stays within the compiled orders.
static double theta_cap(const Tree::Tune& u) {
    double hi = u.theta_hi;
    while (hi > u.theta_lo && p_for_tolerance(u.tol, hi) > FMM_P_MAX) hi -= 0.005;
    return hi;
}

double tune_theta(const Tree::Tune& u) { return u.trial_kind == 2 ? u.theta_trial : u.theta; }

// One AT3b step on the tuner state; returns the N_levels for the next call
// (tune_theta gives the theta).
int tune_step(Tree::Tune& u, double time_s) {
    u.iter++;
    u.win.push_back(time_s);
    int next = u.trial ? u.trial : u.accepted;
    if (u.trial_kind == 0) {
        u.basetime += time_s;
        u.accepted_evals++;
        u.since_move++;
        if (u.wait_up > 0) u.wait_up--;
        if (u.wait_down > 0) u.wait_down--;
        if ((int)u.win.size() > u.window) u.win.erase(u.win.begin());
        if ((int)u.win.size() >= u.window) u.base_min = vmin(u.win);
        if ((int)u.win.size() >= u.window && u.since_move >= u.period) {
            auto allowed = [&](int dd) {
                const int L = u.accepted + dd;
                if (L < 1 || L > u.max_levels) return false;
                return dd > 0 ? u.wait_up == 0 : u.wait_down == 0;
            };
            auto try_nl = [&]() {
                int d = u.nldir;
                if (!allowed(d)) d = -d;
                if (!allowed(d)) return false;
                u.trial = u.accepted + d;
                u.trial_dir = d;
                u.trial_kind = 1;
                return true;
            };
            auto try_theta = [&]() {
                if (!u.theta_on) return false;
                const double hi = theta_cap(u), step = 0.01 * fib(u.fibcount);
                for (int attempt = 0; attempt < 2; ++attempt) {
                    const double c = std::round((u.theta + u.theta_dir * step) * 1e6) / 1e6;
                    if (c >= u.theta_lo - 1e-12 && c <= hi + 1e-12) {
                        u.theta_trial = c;
                        u.trial_kind = 2;
                        return true;
                    }
                    u.theta_dir = -u.theta_dir;
                }
                return false;
            };
            const bool moved = u.next_kind == 2 ? (try_theta() || try_nl()) : (try_nl() || try_theta());
            if (moved) {
                u.win.clear();
                next = u.trial_kind == 1 ? u.trial : u.accepted;
            }
        }
    } else if ((int)u.win.size() >= u.window) {
        const double m = vmin(u.win);
        double spent = 0;
        for (double x : u.win) spent += x;
        const bool theta_move = u.trial_kind == 2;
        if (m < u.base_min) {  // accept the move and keep walking this way
            if (theta_move) u.theta = u.theta_trial;
            else {
                u.accepted = u.trial;
                u.nldir = u.trial_dir;
            }
            u.base_min = m;
            u.basetime += spent;
            u.accepted_evals += (int)u.win.size();
        } else {
            const double cost = std::max(0.0, spent - u.base_min * (double)u.win.size());
            if (theta_move) {
                // Algorithms 2-4: next Fibonacci step, reversed direction; grow the sequence at its end
                if (u.fibcount < u.fiblength) u.fibcount++;
                else {
                    u.fibcount = 1;
                    u.fiblength++;
                }
                u.theta_dir = -u.theta_dir;
            } else {  // the next N_levels move this way waits until its cost fits the cap
                const double avg = u.accepted_evals ? u.basetime / u.accepted_evals : time_s;
                if (u.trial_dir > 0) {
                    u.upcost += cost;
                    const double uptime = (u.upcost + cost) / u.cap - u.basetime;
                    u.wait_up = uptime > 0 ? (int)std::ceil(uptime / std::max(avg, 1e-30)) : 0;
                } else {
                    u.downcost += cost;
                    const double downtime = (u.downcost + cost) / u.cap - u.basetime;
                    u.wait_down = downtime > 0 ? (int)std::ceil(downtime / std::max(avg, 1e-30)) : 0;
                }
                u.nldir = -u.trial_dir;
            }
            u.rejected++;
            u.tuning_cost += cost;
        }
        u.next_kind = theta_move ? 1 : 2;
        u.trial = 0;
        u.trial_kind = 0;
        u.theta_trial = 0;
        u.since_move = 0;
        u.win.clear();
        next = u.accepted;
    }
    return next;
}

}  // namespace fmm

struct fmm_autotuner {
    Tree::Tune u;
};

extern "C" fmm_status fmm_autotune_config(fmm_tree* h, double cap, int window, int period) {
    if (!h || !(cap > 0.0) || window < 1 || period < 1) {
        set_error("autotune_config: need cap > 0, window >= 1, period >= 1");
        return FMM_ERR_INVALID_ARG;
    }
    h->t.tune.cap = cap;
    h->t.tune.window = window;
    h->t.tune.period = period;
    return FMM_OK;
}

extern "C" fmm_status fmm_autotune_step(fmm_tree* h, double time_s, fmm_params* inout) {
    if (!h || !inout || !(time_s >= 0.0)) {
        set_error("autotune_step: NULL argument or negative time");
        return FMM_ERR_INVALID_ARG;
    }
    Tree& t = h->t;
    if (t.batched) {
        set_error("autotune_step: batched trees keep their per-instance N_levels");
        return FMM_ERR_INVALID_ARG;
    }
    if (t.tune.accepted < 1) t.tune.accepted = t.inst_levels[0];
    inout->nlevels = tune_step(t.tune, time_s);
    if (t.tune.theta_on) {
        inout->theta = tune_theta(t.tune);
        inout->p = p_for_tolerance(t.tune.tol, inout->theta);
    } else {
        inout->theta = t.theta;
    }
    return FMM_OK;
}

static bool theta_args_ok(double tol, double lo, double hi) {
    return tol > 0.0 && tol < 1.0 && lo > 0.0 && hi < 1.0 && lo <= hi && p_for_tolerance(tol, lo) <= FMM_P_MAX;
}

extern "C" fmm_status fmm_autotune_theta(fmm_tree* h, double tol, double theta_min, double theta_max) {
    if (!h || !theta_args_ok(tol, theta_min, theta_max)) {
        set_error("autotune_theta: need 0 < tol < 1, 0 < theta_min <= theta_max < 1, p(tol, theta_min) <= 32");
        return FMM_ERR_INVALID_ARG;
    }
    Tree::Tune& u = h->t.tune;
    u.theta_on = true;
    u.tol = tol;
    u.theta_lo = theta_min;
    u.theta_hi = theta_max;
    u.theta = std::min(std::max(h->t.theta, theta_min), theta_cap(u));
    return FMM_OK;
}

extern "C" int fmm_p_for_tolerance(double tol, double theta) { return p_for_tolerance(tol, theta); }

extern "C" fmm_status fmm_autotuner_create(int nlevels, int max_levels, double cap, int window, int period,
                                           fmm_autotuner** out) {
    if (!out || nlevels < 1 || max_levels < nlevels || !(cap > 0.0) || window < 1 || period < 1) {
        set_error("autotuner_create: need 1 <= nlevels <= max_levels, cap > 0, window >= 1, period >= 1");
        return FMM_ERR_INVALID_ARG;
    }
    fmm_autotuner* a = new (std::nothrow) fmm_autotuner();
    if (!a) return FMM_ERR_OOM;
    a->u.accepted = nlevels;
    a->u.max_levels = max_levels;
    a->u.cap = cap;
    a->u.window = window;
    a->u.period = period;
    *out = a;
    return FMM_OK;
}

extern "C" fmm_status fmm_autotuner_step(fmm_autotuner* a, double time_s, int* nlevels_out) {
    if (!a || !nlevels_out || !(time_s >= 0.0)) {
        set_error("autotuner_step: NULL argument or negative time");
        return FMM_ERR_INVALID_ARG;
    }
    *nlevels_out = tune_step(a->u, time_s);
    return FMM_OK;
}

extern "C" fmm_status fmm_autotuner_theta(fmm_autotuner* a, double theta, double tol, double theta_min,
                                          double theta_max) {
    if (!a || !theta_args_ok(tol, theta_min, theta_max) || !(theta >= theta_min && theta <= theta_max) ||
        p_for_tolerance(tol, theta) > FMM_P_MAX) {
        set_error("autotuner_theta: need 0 < tol < 1, 0 < theta_min <= theta <= theta_max < 1, "
                  "p(tol, theta) <= 32");
        return FMM_ERR_INVALID_ARG;
    }
    a->u.theta_on = true;
    a->u.tol = tol;
    a->u.theta_lo = theta_min;
    a->u.theta_hi = theta_max;
    a->u.theta = theta;
    return FMM_OK;
}

extern "C" fmm_status fmm_autotuner_step_params(fmm_autotuner* a, double time_s, int* nlevels_out,
                                                double* theta_out, int* p_out) {
    if (!a || !nlevels_out || !theta_out || !p_out || !(time_s >= 0.0)) {
        set_error("autotuner_step_params: NULL argument or negative time");
        return FMM_ERR_INVALID_ARG;
    }
    *nlevels_out = tune_step(a->u, time_s);
    *theta_out = tune_theta(a->u);
    *p_out = a->u.theta_on ? p_for_tolerance(a->u.tol, *theta_out) : -1;
    return FMM_OK;
}

extern "C" fmm_status fmm_autotuner_stats(const fmm_autotuner* a, double* out, int nout) {
    if (!a || !out) return FMM_ERR_INVALID_ARG;
    const double v[8] = {(double)a->u.accepted, (double)a->u.iter, (double)a->u.rejected, a->u.tuning_cost,
                         a->u.basetime, (double)a->u.trial, a->u.theta, a->u.theta_trial};
    for (int i = 0; i < nout && i < 8; ++i) out[i] = v[i];
    return FMM_OK;
}

extern "C" void fmm_autotuner_destroy(fmm_autotuner* a) { delete a; }
