// N_levels autotuner: Algorithm 4 ("AT3b", Sec. 4.2) of the paper, a directed
// walk in N_levels whose moves that degrade the run time are re-tried only
// after enough accepted evaluations that the accumulated cost of the bad moves
// stays below a user cap on the relative tuning cost.  Noise is filtered as in
// Sec. 4.2.1: every decision compares the minimum time over a short window of
// evaluations.  theta stays fixed (the load-balance variant AT3a has no
// counterpart: the whole evaluation runs on one device).
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

// One AT3b step on the tuner state; returns the N_levels for the next call.
int tune_step(Tree::Tune& u, double time_s) {
    u.iter++;
    u.win.push_back(time_s);
    int next = u.trial ? u.trial : u.accepted;
    if (u.trial == 0) {
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
            int d = u.nldir;
            if (!allowed(d)) d = -d;
            if (allowed(d)) {
                u.trial = u.accepted + d;
                u.trial_dir = d;
                u.win.clear();
                next = u.trial;
            }
        }
    } else if ((int)u.win.size() >= u.window) {
        const double m = vmin(u.win);
        double spent = 0;
        for (double x : u.win) spent += x;
        if (m < u.base_min) {  // accept the move and keep walking this way
            u.accepted = u.trial;
            u.base_min = m;
            u.nldir = u.trial_dir;
            u.basetime += spent;
            u.accepted_evals += (int)u.win.size();
        } else {  // reject: the next move this way waits until its cost fits the cap
            const double cost = std::max(0.0, spent - u.base_min * (double)u.win.size());
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
            u.rejected++;
            u.tuning_cost += cost;
        }
        u.trial = 0;
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
    inout->theta = t.theta;
    return FMM_OK;
}

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

extern "C" fmm_status fmm_autotuner_stats(const fmm_autotuner* a, double* out, int nout) {
    if (!a || !out) return FMM_ERR_INVALID_ARG;
    const double v[6] = {(double)a->u.accepted, (double)a->u.iter, (double)a->u.rejected, a->u.tuning_cost,
                         a->u.basetime, (double)a->u.trial};
    for (int i = 0; i < nout && i < 6; ++i) out[i] = v[i];
    return FMM_OK;
}

extern "C" void fmm_autotuner_destroy(fmm_autotuner* a) { delete a; }
