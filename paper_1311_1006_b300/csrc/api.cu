// C ABI of the FMM library: argument checks, tree life cycle, evaluation
// (eager or replayed from a captured CUDA graph), export and diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "fmm_internal.cuh"

namespace fmm {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

fmm_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FMM_ERR_OOM;
    }
    return FMM_ERR_CUDA;
}

static fmm_status invalid(const std::string& msg) {
    g_err = msg;
    return FMM_ERR_INVALID_ARG;
}

static int max_levels_for(int64_t n) {  // largest N_levels with 4^(L-1) <= n
    int L = 1;
    while (L < 15 && (int64_t(1) << (2 * L)) <= n) ++L;
    return L;
}

// ---- cost model of eqs (2.4)-(2.5) -------------------------------------------
// P2P work  C_P2P = N^2/(2 N_f) * pi ((1+theta)/theta)^2      (eq 2.4)
// M2L work  C_M2L = (3 N_f/2) p^2 * pi ((1+theta)/theta)^2    (eq 2.5)
// With unit costs alpha (time per unit of C_P2P) and beta (per unit of C_M2L),
// alpha C_P2P + beta C_M2L is smallest at N_f* = (N/p) sqrt(alpha/(3 beta)).
// The unit costs are per precision path and process-wide: built-in values
// measured on B300 (1e6-point cluster set, p = 17, theta = 0.5, N_levels = 9,
// P2P and M2L each timed alone), replaced by fmm_cost_model_calibrate from the
// phase times of an evaluation, or set by fmm_cost_model_set.
static std::mutex g_cost_mu;
static double g_alpha[2] = {4.69e-12, 2.34e-10};
static double g_beta[2] = {9.8e-13, 5.5e-11};

static double coupling_area(double theta) {  // pi ((1+theta)/theta)^2
    const double q = (1.0 + theta) / theta;
    return 3.14159265358979323846 * q * q;
}

int seed_nlevels(int64_t n, int p, double alpha, double beta) {
    const int Lmax = max_levels_for(n);
    const double nf = (double)n / (double)std::max(p, 1) * std::sqrt(alpha / (3.0 * beta));
    int best = 1;
    double bestd = 1e300;
    for (int L = 1; L <= Lmax; ++L) {
        const double d = std::fabs(std::log(std::pow(4.0, L - 1) / nf));
        if (d < bestd) {
            bestd = d;
            best = L;
        }
    }
    return best;
}

int default_nlevels(int64_t n, int p, int path) {
    double a, b;
    {
        std::lock_guard<std::mutex> lk(g_cost_mu);
        a = g_alpha[path == FMM_PATH_FP64];
        b = g_beta[path == FMM_PATH_FP64];
    }
    return seed_nlevels(n, p, a, b);
}

static fmm_status check_params(const fmm_params* prm) {
    if (!prm) return invalid("params is NULL");
    if (prm->p < 1 || prm->p > FMM_P_MAX) return invalid("p must be in [1, 32]");
    if (!(prm->theta > 0.0 && prm->theta < 1.0)) return invalid("theta must be in (0, 1)");
    if (prm->path != FMM_PATH_FP32 && prm->path != FMM_PATH_FP64) return invalid("path must be 0 (FP32) or 1 (FP64)");
    if (prm->nlevels < 0) return invalid("nlevels must be >= 0");
    return FMM_OK;
}

static void invalidate_graph(Tree& t) {
    if (t.graph) cudaGraphExecDestroy(t.graph);
    t.graph = nullptr;
    for (auto& k : t.graph_key) k = nullptr;
}

static void apply_params(Tree& t, const fmm_params* prm) {
    t.p = prm->p;
    t.P = compiled_order(prm->p);
    t.PS = (t.P + 2) & ~1;  // >= P+1: slot P holds the constant term of the logarithmic kernel
    t.theta = prm->theta;
    t.path = prm->path;
    t.flags = prm->flags;
}

// Words of the pinned copy of a build's counters: the status word and counters [0, 5), the level bases and
// size requests of the list passes from word 8.
constexpr int kChkWords = 8 + 2 * kMaxLevels + 6;

static fmm_status ensure_streams(Tree& t) {
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    FMM_CUDA(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev));
    // The evaluation forks the far-field chain (a sequence of short, partly
    // latency-bound kernels) onto a high-priority stream and the P2P pass onto
    // a low-priority one, so that far-field blocks are scheduled first as P2P
    // blocks retire.
    int lo_prio = 0, hi_prio = 0;
    FMM_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    if (!t.s_aux) FMM_CUDA(cudaStreamCreateWithPriority(&t.s_aux, cudaStreamNonBlocking, lo_prio));
    if (!t.s_far) FMM_CUDA(cudaStreamCreateWithPriority(&t.s_far, cudaStreamNonBlocking, hi_prio));
    if (!t.s_far2) FMM_CUDA(cudaStreamCreateWithPriority(&t.s_far2, cudaStreamNonBlocking, hi_prio));
    if (!t.ev_join_far2) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_join_far2, cudaEventDisableTiming));
    if (!t.ev_gather) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_gather, cudaEventDisableTiming));
    if (!t.ev_lists) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_lists, cudaEventDisableTiming));
    if (!t.ev_chk) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_chk, cudaEventDisableTiming));
    if (!t.h_chk) FMM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&t.h_chk), kChkWords * sizeof(unsigned long long)));
    if (!t.ev_fork) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_fork, cudaEventDisableTiming));
    if (!t.ev_join) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_join, cudaEventDisableTiming));
    if (!t.ev_join_far) FMM_CUDA(cudaEventCreateWithFlags(&t.ev_join_far, cudaEventDisableTiming));
    for (auto& e : t.ev_t)
        if (!e) FMM_CUDA(cudaEventCreate(&e));
    return FMM_OK;
}

// Lists + work items of a built tree, with the one host synchronisation of a
// build: the first build learns the exact list and item sizes from the device
// counters; a capacity that was too small is grown (25 % slack) and the lists
// are rebuilt.  When the short coordinate sort met a run it does not resolve,
// the tree is rebuilt from d_xy with the full sort (for this tree from then
// on) and *redone is set.
static fmm_status build_lists(Tree& t, cudaStream_t s, const double* d_xy, bool* redone) {
    fmm_status st;
    for (int attempt = 0; attempt < 16; ++attempt) {
        if ((st = run_lists(t, s))) return st;
        unsigned long long hbuf[5] = {0, 0, 0, 0, 0};
        unsigned long long lb[2 * kMaxLevels + 6];
        FMM_CUDA(cudaMemcpyAsync(hbuf, t.d_status, sizeof(hbuf), cudaMemcpyDeviceToHost, s));
        FMM_CUDA(cudaMemcpyAsync(lb, t.d_lvl_base, sizeof(lb), cudaMemcpyDeviceToHost, s));
        FMM_CUDA(cudaStreamSynchronize(s));
        const unsigned bits = (unsigned)(hbuf[0] & 0xffffffffu);
        if ((bits & ST_SORT_RUN) && !(bits & ST_NONFINITE)) {
            t.sort_full = true;
            if (t.s_far) FMM_CUDA(cudaStreamSynchronize(t.s_far));  // work that read the first tree is done
            if ((st = run_tree_build(t, d_xy, s))) return st;
            if (redone) *redone = true;
            continue;
        }
        if (bits & ST_NONFINITE) {
            set_error("non-finite point coordinate");
            return FMM_ERR_NONFINITE;
        }
        if (bits & ST_INTERNAL) {
            set_error("internal index check failed during the tree build");
            return FMM_ERR_CUDA;
        }
        if (bits & ST_TIMEOUT) {
            set_error("a bounded wait in the list build gave up");
            return FMM_ERR_TIMEOUT;
        }
        const bool ovl = bits & (ST_STRONG_OVERFLOW | ST_WEAK_OVERFLOW);
        if (!ovl && !(bits & ST_ITEM_OVERFLOW)) {
            t.h_counts[0] = lb[t.Lmax];
            t.h_counts[1] = lb[kMaxLevels + t.Lmax];
            t.h_counts[2] = hbuf[3];
            t.h_counts[3] = hbuf[4];
            return FMM_OK;
        }
        const unsigned long long* need = lb + 2 * kMaxLevels;
        auto grow = [](long long cur, unsigned long long want) {
            return std::max<long long>(2 * cur, (long long)(want + want / 4 + 1024));
        };
        if (need[0] > (unsigned long long)t.cand_cap) t.cand_cap = grow(t.cand_cap, need[0]);
        if (need[1] > (unsigned long long)t.scap_tot) t.scap_tot = grow(t.scap_tot, need[1]);
        if (need[2] > (unsigned long long)t.wcap_tot) t.wcap_tot = grow(t.wcap_tot, need[2]);
        if (!ovl && (bits & ST_ITEM_OVERFLOW)) {
            // the item counts, moved aside by k_m2l_rows (the counters themselves are zeroed)
            const unsigned long long ip = need[4], im = need[5];
            if ((long long)ip > t.p2p_cap) t.p2p_cap = (long long)(ip + ip / 4 + 1024);
            if ((long long)im > t.m2l_cap) t.m2l_cap = (long long)(im + im / 4 + 1024);
        }
        if (t.scap_tot >= (1ll << 31) || t.wcap_tot >= (1ll << 31)) {
            set_error("coupling lists exceed 2^31 entries");
            return FMM_ERR_OOM;
        }
        invalidate_graph(t);
        if ((st = alloc_lists(t))) return st;
        FMM_CUDA(cudaMemsetAsync(t.d_status, 0, sizeof(unsigned), s));
    }
    set_error("coupling lists kept overflowing");
    return FMM_ERR_OOM;
}

// Tree build + lists + work items.
static fmm_status build_all(Tree& t, const double* d_xy, cudaStream_t s) {
    fmm_status st = run_tree_build(t, d_xy, s);
    if (st) return st;
    return build_lists(t, s, d_xy, nullptr);
}

static fmm_status shape_and_build(Tree& t, const double* d_xy, cudaStream_t s, bool reshape) {
    fmm_status st;
    if (reshape) {
        invalidate_graph(t);
        if ((st = build_shape(t))) return st;
        if ((st = alloc_build(t))) return st;
        t.eval_nbox = 0;  // force the workspace to follow the new shape
    }
    if ((st = ensure_streams(t))) return st;
    return build_all(t, d_xy, s);
}

static void release(Tree* t) {
    if (!t) return;
    invalidate_graph(*t);
    void* ptrs[] = {t->d_bstart, t->d_bcount, t->d_parent, t->d_child0, t->d_fold_par, t->d_inst, t->d_inst_ptoff,
                    t->d_inst_boxoff, t->d_leaf_start, t->d_inst_levels, t->d_loc, t->d_X2, t->d_Y2, t->d_sideX, t->d_sideY, t->d_part_stat,
                    t->d_sort_hist, t->d_sort_tot, t->d_sort_off, t->d_sort_os, t->d_perm,
                    t->d_leaf_of, t->d_pts, t->d_pos4, t->d_center, t->d_radius, t->d_rho, t->d_chl, t->d_rho32,
                    t->d_rad32, t->d_soff, t->d_ns, t->d_sidx, t->d_srng, t->d_sowner, t->d_ltstat,
                    t->d_lvl_base, t->d_woff, t->d_nw, t->d_widx, t->d_p2p_items,
                    t->d_m2l_items, t->d_m2l_rows, t->d_p2p_rows, t->d_box_tail, t->d_m2l_rowctr, t->d_leaf_items, t->d_box_m2l, t->d_status, t->d_gam, t->d_near, t->d_M64,
                    t->d_pslot, t->d_posp, t->d_slot_of, t->d_gamp, t->d_xy_all, t->d_gam_all, t->d_phi_all,
                    t->d_M32, t->d_Lm2l, t->d_L64, t->d_L32, t->d_p2p_part, t->d_m2l_part, t->d_pstage,
                    t->d_pers, t->d_gamp2, t->d_nsrc};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < 4; ++i) {
        if (t->d_keys[i]) cudaFree(t->d_keys[i]);
        if (t->d_vals[i]) cudaFree(t->d_vals[i]);
    }
    for (auto& l : t->level_boxes)
        if (l.d_ids) cudaFree(l.d_ids);
    for (auto& l : t->level_parents)
        if (l.d_ids) cudaFree(l.d_ids);
    if (t->leaves.d_ids) cudaFree(t->leaves.d_ids);
    for (auto& s : t->seg_x) {
        if (s.d_start) cudaFree(s.d_start);
        if (s.d_nzero) cudaFree(s.d_nzero);
        if (s.d_obefore) cudaFree(s.d_obefore);
    }
    for (auto& s : t->seg_y) {
        if (s.d_start) cudaFree(s.d_start);
        if (s.d_nzero) cudaFree(s.d_nzero);
        if (s.d_obefore) cudaFree(s.d_obefore);
    }
    if (t->s_aux) cudaStreamDestroy(t->s_aux);
    if (t->s_far) cudaStreamDestroy(t->s_far);
    if (t->s_far2) cudaStreamDestroy(t->s_far2);
    if (t->ev_join_far2) cudaEventDestroy(t->ev_join_far2);
    if (t->ev_gather) cudaEventDestroy(t->ev_gather);
    if (t->ev_lists) cudaEventDestroy(t->ev_lists);
    if (t->ev_chk) cudaEventDestroy(t->ev_chk);
    if (t->h_chk) cudaFreeHost(t->h_chk);
    if (t->ev_join_far) cudaEventDestroy(t->ev_join_far);
    if (t->ev_fork) cudaEventDestroy(t->ev_fork);
    if (t->ev_join) cudaEventDestroy(t->ev_join);
    for (auto e : t->ev_t)
        if (e) cudaEventDestroy(e);
}

static fmm_status check_pending() {
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "earlier asynchronous work");
    }
    return FMM_OK;
}

}  // namespace fmm

using namespace fmm;


extern "C" {

const char* fmm_status_string(fmm_status s) {
    switch (s) {
        case FMM_OK: return "ok";
        case FMM_ERR_INVALID_ARG: return "invalid argument";
        case FMM_ERR_CUDA: return "CUDA error";
        case FMM_ERR_OOM: return "out of memory";
        case FMM_ERR_TIMEOUT: return "device wait timed out";
        case FMM_ERR_NONFINITE: return "non-finite input";
    }
    return "unknown status";
}

const char* fmm_last_error(void) { return g_err.c_str(); }

int fmm_default_nlevels(int64_t n, int p, int path) { return n < 1 ? 0 : default_nlevels(n, p, path); }

int fmm_seed_nlevels(int64_t n, int p, double alpha, double beta) {
    if (n < 1 || p < 1 || !(alpha > 0.0) || !(beta > 0.0)) return 0;
    return seed_nlevels(n, p, alpha, beta);
}

fmm_status fmm_cost_model_get(int path, double* alpha, double* beta) {
    if ((path != FMM_PATH_FP32 && path != FMM_PATH_FP64) || !alpha || !beta) return invalid("bad path or NULL");
    std::lock_guard<std::mutex> lk(g_cost_mu);
    *alpha = g_alpha[path];
    *beta = g_beta[path];
    return FMM_OK;
}

fmm_status fmm_cost_model_set(int path, double alpha, double beta) {
    if (path != FMM_PATH_FP32 && path != FMM_PATH_FP64) return invalid("path must be 0 (FP32) or 1 (FP64)");
    if (!(alpha > 0.0) || !(beta > 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
        return invalid("alpha and beta must be finite and > 0");
    std::lock_guard<std::mutex> lk(g_cost_mu);
    g_alpha[path] = alpha;
    g_beta[path] = beta;
    return FMM_OK;
}

fmm_status fmm_cost_model_calibrate(fmm_tree* h, double* alpha_out, double* beta_out) {
    if (!h) return invalid("NULL tree");
    Tree& t = h->t;
    if (!t.timing_valid) return invalid("no evaluation with FMM_FLAG_TIMING yet");
    double ms[7];
    fmm_status st = fmm_phase_times(h, ms, 7);
    if (st) return st;
    // model counts of eqs (2.4)-(2.5), summed over the instances of the tree
    const double area = coupling_area(t.theta);
    double c_p2p = 0.0, c_m2l = 0.0;
    for (int b = 0; b < t.ninst; ++b) {
        const double nb = (double)(t.inst_pt_off[b + 1] - t.inst_pt_off[b]);
        const double nf = std::pow(4.0, t.inst_levels[b] - 1);
        c_p2p += nb * nb / (2.0 * nf) * area;
        if (t.inst_levels[b] >= 3) c_m2l += 1.5 * nf * (double)t.p * (double)t.p * area;
    }
    const double tp = ms[4] * 1e-3, tm = ms[2] * 1e-3;
    if (!(c_m2l > 0.0) || !(tp > 0.0) || !(tm > 0.0))
        return invalid("calibration needs an evaluation with P2P and M2L work (N_levels >= 3)");
    const double a = tp / c_p2p, be = tm / c_m2l;
    if ((st = fmm_cost_model_set(t.path, a, be))) return st;
    if (alpha_out) *alpha_out = a;
    if (beta_out) *beta_out = be;
    return FMM_OK;
}

static fmm_status build_common(const double* d_xy, const std::vector<int64_t>& offs, const fmm_params* prm,
                               const int* h_nlevels, bool batched, void* stream, fmm_tree** out,
                               int64_t n_src = 0) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    fmm_status st = check_params(prm);
    if (st) return st;
    if (!d_xy) return invalid("d_xy is NULL");
    const int B = (int)offs.size() - 1;
    if (B < 1) return invalid("no instance");
    if (offs[0] != 0) return invalid("offsets must start at 0");
    for (int b = 0; b < B; ++b)
        if (offs[b + 1] - offs[b] < 1) return invalid("every instance needs >= 1 point");
    if (offs[B] >= (int64_t(1) << 31) - 1) return invalid("n must be < 2^31");
    if ((st = check_pending())) return st;
    fmm_tree* h = new (std::nothrow) fmm_tree();
    if (!h) return FMM_ERR_OOM;
    Tree& t = h->t;
    apply_params(t, prm);
    t.batched = batched;
    t.n = offs[B];
    t.n_src = n_src;  // separate evaluation points: the first n_src points are the sources
    t.n_tgt = n_src > 0 ? offs[B] - n_src : 0;
    t.ninst = B;
    t.inst_pt_off = offs;
    t.inst_levels.resize(B);
    for (int b = 0; b < B; ++b) {
        const int64_t nb = offs[b + 1] - offs[b];
        int L = h_nlevels ? h_nlevels[b] : prm->nlevels;
        if (L == 0) L = default_nlevels(nb, prm->p, prm->path);
        if (L < 1 || L > max_levels_for(nb)) {
            delete h;
            return invalid("nlevels out of range: need 1 <= nlevels and 4^(nlevels-1) <= points of the instance");
        }
        t.inst_levels[b] = L;
    }
    st = shape_and_build(t, d_xy, static_cast<cudaStream_t>(stream), true);
    if (st) {
        release(&h->t);
        delete h;
        return st;
    }
    t.tune.accepted = t.inst_levels[0];
    t.tune.max_levels = max_levels_for(t.n);
    *out = h;
    return FMM_OK;
}

fmm_status fmm_build_tree(const double* d_xy, int64_t n, const fmm_params* prm, void* stream, fmm_tree** out) {
    if (n < 1) return invalid("n must be >= 1");
    std::vector<int64_t> offs = {0, n};
    return build_common(d_xy, offs, prm, nullptr, false, stream, out);
}

fmm_status fmm_build_tree_batched(const double* d_xy, const int64_t* h_offsets, int B, const fmm_params* prm,
                                  const int* h_nlevels, void* stream, fmm_tree** out) {
    if (!h_offsets || B < 1) return invalid("offsets NULL or B < 1");
    std::vector<int64_t> offs(h_offsets, h_offsets + B + 1);
    return build_common(d_xy, offs, prm, h_nlevels, true, stream, out);
}

// ---- separate evaluation points (eq 2.2) ----------------------------------
// The tree is built over the sources followed by the evaluation points, which
// carry zero strength: a zero-strength point changes no expansion and no near
// sum, and the coincidence rule z_j != z_i of the P2P pass is eq (2.2)'s
// x_j != y_i.  The evaluation gathers the potentials of the evaluation points.

static fmm_status concat_points(Tree& t, const double* d_src, const double* d_tgt, cudaStream_t s) {
    FMM_CUDA(cudaMemcpyAsync(t.d_xy_all, d_src, (size_t)t.n_src * 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    FMM_CUDA(cudaMemcpyAsync(t.d_xy_all + 2 * t.n_src, d_tgt, (size_t)t.n_tgt * 2 * sizeof(double),
                             cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}

fmm_status fmm_build_tree_targets(const double* d_src_xy, int64_t n_src, const double* d_tgt_xy, int64_t n_tgt,
                                  const fmm_params* prm, void* stream, fmm_tree** out) {
    if (!d_src_xy || !d_tgt_xy || !out) return invalid("NULL argument");
    if (n_src < 1 || n_tgt < 1) return invalid("n_src and n_tgt must be >= 1");
    const int64_t n = n_src + n_tgt;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc((void**)&buf, (size_t)n * 2 * sizeof(double));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error("device allocation failed (points)");
        return FMM_ERR_OOM;
    }
    FMM_CUDA(e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(buf, d_src_xy, (size_t)n_src * 2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf + 2 * n_src, d_tgt_xy, (size_t)n_tgt * 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                            s);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "cudaMemcpyAsync(points)");
    }
    std::vector<int64_t> offs = {0, n};
    const fmm_status st = build_common(buf, offs, prm, nullptr, false, stream, out, n_src);
    if (st) {
        cudaFree(buf);
        return st;
    }
    Tree& t = (*out)->t;
    t.d_xy_all = buf;
    t.n_src = n_src;
    t.n_tgt = n_tgt;
    return FMM_OK;
}

fmm_status fmm_tree_rebuild_targets(fmm_tree* h, const double* d_src_xy, const double* d_tgt_xy,
                                    const fmm_params* prm, void* stream) {
    if (!h || !d_src_xy || !d_tgt_xy) return invalid("NULL argument");
    Tree& t = h->t;
    if (t.n_src == 0) return invalid("not a tree with separate evaluation points (fmm_build_tree_targets)");
    fmm_status st;
    if ((st = concat_points(t, d_src_xy, d_tgt_xy, static_cast<cudaStream_t>(stream)))) return st;
    return fmm_tree_rebuild(h, t.d_xy_all, prm, stream);
}

static fmm_status eval_common(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream);

static fmm_status eval_targets_common(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream,
                                      bool log_kernel) {
    if (!h || !d_gamma || !d_phi) return invalid("NULL argument");
    Tree& t = h->t;
    if (t.n_src == 0) return invalid("not a tree with separate evaluation points (fmm_build_tree_targets)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t cs = t.path == FMM_PATH_FP32 ? 8 : 16;
    if (!t.d_gam_all) {
        FMM_CUDA(cudaMalloc((void**)&t.d_gam_all, (size_t)t.n * 2 * sizeof(double)));
        FMM_CUDA(cudaMemset(t.d_gam_all, 0, (size_t)t.n * 2 * sizeof(double)));  // evaluation points: strength 0
    }
    if (t.phi_all_path != t.path) {
        if (t.d_phi_all) cudaFree(t.d_phi_all);
        t.d_phi_all = nullptr;
        FMM_CUDA(cudaMalloc(&t.d_phi_all, (size_t)t.n * cs));
        t.phi_all_path = t.path;
    }
    FMM_CUDA(cudaMemcpyAsync(t.d_gam_all, d_gamma, (size_t)t.n_src * 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                             s));
    fmm_status st = log_kernel ? fmm_eval_log(h, t.d_gam_all, t.d_phi_all, stream)
                               : eval_common(h, t.d_gam_all, t.d_phi_all, stream);
    if (st) return st;
    FMM_CUDA(cudaMemcpyAsync(d_phi, static_cast<char*>(t.d_phi_all) + (size_t)t.n_src * cs, (size_t)t.n_tgt * cs,
                             cudaMemcpyDeviceToDevice, s));
    return FMM_OK;
}

fmm_status fmm_eval_targets(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream) {
    return eval_targets_common(h, d_gamma, d_phi, stream, false);
}

fmm_status fmm_eval_targets_log(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream) {
    return eval_targets_common(h, d_gamma, d_phi, stream, true);
}

fmm_status fmm_tree_rebuild(fmm_tree* h, const double* d_xy, const fmm_params* prm, void* stream) {
    if (!h || !d_xy) return invalid("NULL argument");
    Tree& t = h->t;
    fmm_status st;
    if ((st = check_pending())) return st;
    bool reshape = false;
    if (prm) {
        if ((st = check_params(prm))) return st;
        if (!t.batched && prm->nlevels != 0 && prm->nlevels != t.inst_levels[0]) {
            if (prm->nlevels > max_levels_for(t.n)) return invalid("nlevels out of range");
            t.inst_levels[0] = prm->nlevels;
            reshape = true;
        }
        if (prm->p != t.p || prm->path != t.path) t.eval_nbox = 0;
        if (prm->theta != t.theta || prm->p != t.p || prm->path != t.path) invalidate_graph(t);
        const int old_flags = t.flags;
        apply_params(t, prm);
        if (old_flags != t.flags) invalidate_graph(t);
    }
    return shape_and_build(t, d_xy, static_cast<cudaStream_t>(stream), reshape);
}

// Rebuild + evaluate in one call.  The upward pass (strength gather, P2M,
// M2M) needs the tree but not the coupling lists, so it runs on the far-field
// stream while the lists are built on the caller's stream; the downward pass
// follows on the far-field stream and P2P on the low-priority stream, as in
// fmm_eval, queued behind the lists on the device once an earlier build has
// sized the capacities (else after the build's host check).  Same kernels in
// the same per-stream order as fmm_tree_rebuild + fmm_eval, so the same result
// bit for bit.
fmm_status fmm_step(fmm_tree* h, const double* d_xy, const double* d_gamma, void* d_phi, void* stream) {
    if (!h || !d_xy || !d_gamma || !d_phi) return invalid("NULL argument");
    Tree& t = h->t;
    if (t.n_src > 0) return invalid("tree with separate evaluation points: use fmm_tree_rebuild_targets + fmm_eval_targets");
    fmm_status st;
    if (t.batched || (t.flags & (FMM_FLAG_SERIAL | FMM_FLAG_TIMING | FMM_FLAG_GRAPH | FMM_FLAG_PERSISTENT))) {
        // phase timing, the serial order and graph replay are defined on the two-call sequence
        if ((st = fmm_tree_rebuild(h, d_xy, nullptr, stream))) return st;
        return t.batched ? fmm_eval_batched(h, d_gamma, d_phi, stream) : fmm_eval(h, d_gamma, d_phi, stream);
    }
    if ((st = check_pending())) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = ensure_streams(t))) return st;
    if (t.h_counts[0] != 0 && t.grid_p2p_items > 0 && t.grid_m2l_items > 0) {
        // Capacities and launch grids known from an earlier build: the evaluation is queued behind the list
        // passes on the device, and the host checks the build's counters (copied after the lists) while it
        // runs.  A build that overflowed a capacity, gave up a wait, met a non-finite coordinate or a long
        // run of equal sort keys, or needs larger grids, is done again in the checked order below; the
        // evaluation queued behind it did only in-bounds work on stale tables (no items after an overflow).
        if ((st = run_tree_build(t, d_xy, s))) return st;
        const unsigned gen0 = t.eval_gen;
        if ((st = alloc_eval_core(t, 1))) return st;
        if ((st = alloc_eval_parts(t))) return st;
        if (t.eval_gen != gen0) invalidate_graph(t);  // a captured evaluation holds the old buffers
        const Bufs B = bufs(t, 0);
        t.p2p_funcs.clear();
        FMM_CUDA(cudaEventRecord(t.ev_fork, s));
        FMM_CUDA(cudaStreamWaitEvent(t.s_far, t.ev_fork, 0));
        launch_gather(t, B, d_gamma, t.s_far);
        FMM_CUDA(cudaEventRecord(t.ev_gather, t.s_far));
        dispatch_up(t, B, t.s_far);
        if ((st = run_lists(t, s))) return st;
        FMM_CUDA(cudaEventRecord(t.ev_lists, s));
        FMM_CUDA(cudaMemcpyAsync(t.h_chk, t.d_status, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        FMM_CUDA(cudaMemcpyAsync(t.h_chk + 8, t.d_lvl_base, (2 * kMaxLevels + 6) * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
        FMM_CUDA(cudaEventRecord(t.ev_chk, s));
        FMM_CUDA(cudaStreamWaitEvent(t.s_far, t.ev_lists, 0));
        dispatch_down(t, B, t.s_far);
        FMM_CUDA(cudaEventRecord(t.ev_join_far, t.s_far));
        FMM_CUDA(cudaStreamWaitEvent(t.s_aux, t.ev_gather, 0));
        FMM_CUDA(cudaStreamWaitEvent(t.s_aux, t.ev_lists, 0));
        launch_near(t, B, t.s_aux);
        FMM_CUDA(cudaEventRecord(t.ev_join, t.s_aux));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join_far, 0));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
        launch_l2p_near(t, B, d_phi, s);
        FMM_CUDA(cudaGetLastError());
        t.timing_valid = false;
        FMM_CUDA(cudaEventSynchronize(t.ev_chk));
        const unsigned bits = (unsigned)(t.h_chk[0] & 0xffffffffu);
        const unsigned long long* lb = t.h_chk + 8;
        const bool ok = !(bits & (ST_NONFINITE | ST_STRONG_OVERFLOW | ST_WEAK_OVERFLOW | ST_TIMEOUT | ST_INTERNAL |
                                  ST_ITEM_OVERFLOW | ST_SORT_RUN)) &&
                        (long long)t.h_chk[3] <= t.grid_p2p_items && (long long)t.h_chk[4] <= t.grid_m2l_items;
        if (ok) {
            t.h_counts[0] = lb[t.Lmax];
            t.h_counts[1] = lb[kMaxLevels + t.Lmax];
            t.h_counts[2] = t.h_chk[3];
            t.h_counts[3] = t.h_chk[4];
            if (refresh_grids(t)) invalidate_graph(t);  // grids for the next evaluation
            return FMM_OK;
        }
        FMM_CUDA(cudaStreamSynchronize(s));  // the queued evaluation is done; the checked order replaces its result
    }
    if ((st = run_tree_build(t, d_xy, s))) return st;
    const unsigned gen = t.eval_gen;
    if ((st = alloc_eval_core(t, 1))) return st;
    const Bufs B = bufs(t, 0);
    t.p2p_funcs.clear();
    FMM_CUDA(cudaEventRecord(t.ev_fork, s));
    FMM_CUDA(cudaStreamWaitEvent(t.s_far, t.ev_fork, 0));
    launch_gather(t, B, d_gamma, t.s_far);
    FMM_CUDA(cudaEventRecord(t.ev_gather, t.s_far));
    dispatch_up(t, B, t.s_far);
    bool redone = false;
    if ((st = build_lists(t, s, d_xy, &redone))) return st;  // host check; the upward pass runs meanwhile
    if (redone) {  // the tree was built again (full coordinate sort): its gather and upward pass again
        FMM_CUDA(cudaEventRecord(t.ev_fork, s));
        FMM_CUDA(cudaStreamWaitEvent(t.s_far, t.ev_fork, 0));
        launch_gather(t, B, d_gamma, t.s_far);
        FMM_CUDA(cudaEventRecord(t.ev_gather, t.s_far));
        dispatch_up(t, B, t.s_far);
    }
    // the partial-sum buffers follow the list capacities just learned: allocate them now and take the
    // buffer table again (the one above predates them)
    if ((st = alloc_eval_parts(t))) return st;
    const bool regrid = refresh_grids(t);  // always: the grids must cover this build's item counts
    if (t.eval_gen != gen || regrid) invalidate_graph(t);
    const Bufs Bd = bufs(t, 0);
    dispatch_down(t, Bd, t.s_far);
    FMM_CUDA(cudaEventRecord(t.ev_join_far, t.s_far));
    FMM_CUDA(cudaStreamWaitEvent(t.s_aux, t.ev_gather, 0));  // slot-layout strengths; the lists are complete
    launch_near(t, Bd, t.s_aux);
    FMM_CUDA(cudaEventRecord(t.ev_join, t.s_aux));
    FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join_far, 0));
    FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
    launch_l2p_near(t, Bd, d_phi, s);
    FMM_CUDA(cudaGetLastError());
    t.timing_valid = false;
    return FMM_OK;
}

fmm_status fmm_eval_status(fmm_tree* h, void* stream) {
    if (!h) return invalid("NULL tree");
    Tree& t = h->t;
    if (!t.d_status) return FMM_OK;
    unsigned bits = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FMM_CUDA(cudaMemcpyAsync(&bits, t.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    if (bits & ST_TIMEOUT) {
        unsigned long long stage = 0;
        if (t.d_pers) {
            FMM_CUDA(cudaMemcpyAsync(&stage, t.d_pers + 3, sizeof(stage), cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaStreamSynchronize(s));
        }
        set_error(stage ? "a work-queue wait of the persistent evaluation ran out (stage " + std::to_string(stage - 1) +
                              ")"
                        : std::string("a bounded wait of the evaluation ran out"));
        return FMM_ERR_TIMEOUT;
    }
    if (bits & ST_INTERNAL) {
        set_error("an internal check of the evaluation failed");
        return FMM_ERR_CUDA;
    }
    return FMM_OK;
}

fmm_status fmm_selftest_bounded_wait(int which, void* stream) {
    if (which < 0 || which > 2) return invalid("which must be 0 (look-back), 1 (mbarrier) or 2 (work queue)");
    fmm_status st;
    if ((st = check_pending())) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long* buf = nullptr;  // [0] status word, [1..2] tile status words
    FMM_CUDA(cudaMalloc((void**)&buf, 4 * sizeof(unsigned long long)));
    cudaError_t e = cudaMemsetAsync(buf, 0, 4 * sizeof(unsigned long long), s);
    unsigned* status = reinterpret_cast<unsigned*>(buf);
    if (e == cudaSuccess) {
        if (which == 0) launch_selftest_lookback(buf + 1, 1 << 12, status, s);
        else if (which == 1) launch_selftest_mbar(1 << 12, status, s);
        else launch_selftest_queue(buf, 20000000ull, status, s);  // 20 ms; [1], [2] counters, [3] stage
        e = cudaGetLastError();
    }
    unsigned h_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    FMM_CUDA(e);
    if (h_status & ST_TIMEOUT) {
        set_error("a bounded device wait ran out (self-test)");
        return FMM_ERR_TIMEOUT;
    }
    return FMM_OK;
}

fmm_status fmm_selftest_rcp64(const double* d_x, double* d_out, int64_t n, void* stream) {
    if (!d_x || !d_out || n < 0) return invalid("NULL argument or n < 0");
    if (n == 0) return FMM_OK;
    launch_selftest_rcp64(d_x, n, d_out, static_cast<cudaStream_t>(stream));
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

void fmm_tree_destroy(fmm_tree* h) {
    if (!h) return;
    release(&h->t);
    delete h;
}

// Stream priorities of the evaluation (far field high, P2P low) set on the
// captured kernel nodes, which otherwise run at the priority of the stream the
// graph is launched into.  Best effort: a node that refuses keeps the default.
static void set_node_priorities(const Tree& t, cudaGraph_t g) {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return;
    }
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        const bool p2p = std::find(t.p2p_funcs.begin(), t.p2p_funcs.end(), kp.func) != t.p2p_funcs.end();
        cudaLaunchAttributeValue v{};
        v.priority = p2p ? lo : hi;
        cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v);
    }
    cudaGetLastError();
}

// Evaluation workspace of `sets` strength sets; a reallocation invalidates the
// captured graph, whose nodes hold the old buffer addresses.
static fmm_status ensure_eval(Tree& t, int sets) {
    const unsigned gen = t.eval_gen;
    const fmm_status st = alloc_eval(t, sets);
    if (st || t.eval_gen != gen) invalidate_graph(t);
    if (!st && refresh_grids(t)) invalidate_graph(t);
    return st;
}

static fmm_status eval_common(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream) {
    if (!h || !d_gamma || !d_phi) return invalid("NULL argument");
    Tree& t = h->t;
    fmm_status st;
    if ((st = check_pending())) return st;
    if (t.eval_nbox == 0) invalidate_graph(t);
    if ((st = ensure_eval(t, 1))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool use_graph =
        (t.flags & FMM_FLAG_GRAPH) && !(t.flags & (FMM_FLAG_NO_GRAPH | FMM_FLAG_TIMING)) && s != nullptr;
    const bool persistent = t.flags & FMM_FLAG_PERSISTENT;
    if (persistent && (st = prepare_persistent(t))) return st;  // table upload: before any capture
    auto run = [&]() { return persistent ? run_eval_persistent(t, d_gamma, d_phi, s) : run_eval(t, d_gamma, d_phi, s); };
    if (!use_graph) return run();
    const void* key[4] = {d_gamma, d_phi, (const void*)s, (const void*)(intptr_t)(t.path * 64 + t.P)};
    if (!t.graph || memcmp(key, t.graph_key, sizeof(key)) != 0) {
        invalidate_graph(t);
        FMM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = run();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        FMM_CUDA(e);
        set_node_priorities(t, g);
        e = cudaGraphInstantiate(&t.graph, g, 0);
        cudaGraphDestroy(g);
        FMM_CUDA(e);
        memcpy(t.graph_key, key, sizeof(key));
    }
    FMM_CUDA(cudaGraphLaunch(t.graph, s));
    return FMM_OK;
}

fmm_status fmm_eval(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream) {
    return eval_common(h, d_gamma, d_phi, stream);
}

fmm_status fmm_eval_log(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream) {
    if (!h || !d_gamma || !d_phi) return invalid("NULL argument");
    Tree& t = h->t;
    fmm_status st;
    if ((st = check_pending())) return st;
    if ((st = ensure_eval(t, 2))) return st;
    return run_eval_log(t, d_gamma, d_phi, static_cast<cudaStream_t>(stream));
}

fmm_status fmm_eval_batched(fmm_tree* h, const double* d_gamma, void* d_phi, void* stream) {
    if (h && !h->t.batched) return invalid("tree was not built by fmm_build_tree_batched");
    return eval_common(h, d_gamma, d_phi, stream);
}

fmm_status fmm_eval_backward(fmm_tree* h, const double* d_gamma, const double* d_gphi, double* d_ggamma,
                             double* d_gxy, void* stream) {
    if (!h || !d_gamma || !d_gphi) return invalid("NULL argument");
    if (!d_ggamma && !d_gxy) return FMM_OK;
    Tree& t = h->t;
    if (t.n_src > 0) return invalid("the adjoint is defined for trees without separate evaluation points");
    fmm_status st;
    if ((st = check_pending())) return st;
    if ((st = ensure_eval(t, 2))) return st;
    return run_backward(t, d_gamma, d_gphi, d_ggamma, d_gxy, static_cast<cudaStream_t>(stream));
}

fmm_status fmm_phase_times(fmm_tree* h, double* out, int nout) {
    if (!h || !out || nout < 1) return invalid("NULL argument");
    Tree& t = h->t;
    if (!t.timing_valid) return invalid("no evaluation with FMM_FLAG_TIMING yet");
    FMM_CUDA(cudaEventSynchronize(t.ev_t[7]));
    float ms[7] = {0, 0, 0, 0, 0, 0, 0};
    FMM_CUDA(cudaEventElapsedTime(&ms[0], t.ev_t[0], t.ev_t[1]));
    FMM_CUDA(cudaEventElapsedTime(&ms[1], t.ev_t[1], t.ev_t[2]));
    FMM_CUDA(cudaEventElapsedTime(&ms[2], t.ev_t[2], t.ev_t[3]));
    FMM_CUDA(cudaEventElapsedTime(&ms[3], t.ev_t[3], t.ev_t[4]));
    FMM_CUDA(cudaEventElapsedTime(&ms[4], t.ev_t[5], t.ev_t[6]));
    FMM_CUDA(cudaEventElapsedTime(&ms[5], t.ev_t[8], t.ev_t[7]));
    FMM_CUDA(cudaEventElapsedTime(&ms[6], t.ev_t[0], t.ev_t[7]));
    for (int i = 0; i < nout && i < 7; ++i) out[i] = ms[i];
    return FMM_OK;
}

fmm_status fmm_get_tree_info(const fmm_tree* h, fmm_tree_info* out) {
    if (!h || !out) return invalid("NULL argument");
    const Tree& t = h->t;
    out->n = t.n;
    out->ninst = t.ninst;
    out->nlevels_max = t.Lmax;
    out->p = t.p;
    out->path = t.path;
    out->theta = t.theta;
    out->nboxes = t.nbox;
    out->nleaves = t.nleaf;
    unsigned long long c[2] = {0, 0};
    fmm_status st = run_count(const_cast<Tree&>(t), nullptr, c);
    if (st) return st;
    out->n_strong = (int64_t)t.h_counts[0];
    out->n_weak = (int64_t)t.h_counts[1];
    out->n_strong_leaf = (int64_t)c[0];
    out->p2p_pairs = (int64_t)c[1];
    out->p2p_items = (int64_t)t.h_counts[2];
    out->m2l_items = (int64_t)t.h_counts[3];
    out->autotune_nlevels = t.tune.accepted;
    const int lv = t.Lmax - 1;
    const int lg = std::min(t.l0, lv);
    // kernels per build: coordinate sort (see below), first cut flags 1 (written by the short sort instead),
    // per global level 2 partitions (the x cut also computes that level's geometry), the geometry of the last
    // globally split level 1, subtree 1, finalize 1, lists root 1 + one pass per level, items 1, M2L row
    // order 1; batched: instance keys 1 + 2 sort passes x 3.  Sort: digit counts + 4 passes + runs (short),
    // counts + 8 passes (full), beyond 2^30 points keys + 8 x 3.
    const bool big = t.n >= (1 << 30), full = t.sort_full || t.ninst > 1;
    const int sortk = big ? 25 : (full ? 9 : 6);
    const int mark = lg > 0 && (big || full) ? 1 : 0;
    out->launches_build = 5 + sortk + lv + 2 * lg + mark + (lg < lv ? 1 : 0) + (t.ninst > 1 ? 7 : 0);
    // per evaluation: gather, P2M, M2M per level, M2L, M2L partial sums, L2L per level (not the deepest on
    // the FP32 path), P2P, L2P (which adds the P2P partial sums of split leaves)
    out->launches_eval = 6 + 2 * lv - (fold_leaf_l2l(t) ? 1 : 0);
    out->autotune_theta = t.tune.theta_on ? t.tune.theta : t.theta;
    return FMM_OK;
}

fmm_status fmm_tree_export(const fmm_tree* h, int what, void* h_dst, int64_t count, void* stream) {
    if (!h || !h_dst) return invalid("NULL argument");
    const Tree& t = h->t;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = t.n, nb = t.nbox;
    auto copy = [&](const void* src, int64_t elems, size_t esz) -> fmm_status {
        if (count < elems) return invalid("host buffer too small");
        if (!src) return invalid("array not available (no evaluation yet?)");
        FMM_CUDA(cudaMemcpyAsync(h_dst, src, (size_t)elems * esz, cudaMemcpyDeviceToHost, s));
        FMM_CUDA(cudaStreamSynchronize(s));
        return FMM_OK;
    };
    switch (what) {
        case FMM_EXPORT_PERM: return copy(t.d_perm, n, 4);
        case FMM_EXPORT_BSTART: return copy(t.d_bstart, nb, 4);
        case FMM_EXPORT_BCOUNT: return copy(t.d_bcount, nb, 4);
        case FMM_EXPORT_CENTER: return copy(t.d_center, 2 * nb, 8);
        case FMM_EXPORT_RADIUS: return copy(t.d_radius, nb, 8);
        case FMM_EXPORT_RHO: return copy(t.d_rho, nb, 8);
        case FMM_EXPORT_NSTRONG:
        case FMM_EXPORT_NWEAK: {  // the device keeps each list's end: length = end - first entry
            const bool strong = what == FMM_EXPORT_NSTRONG;
            fmm_status st = copy(strong ? t.d_ns : t.d_nw, nb, 4);
            if (st) return st;
            std::vector<int32_t> off((size_t)nb);
            FMM_CUDA(cudaMemcpyAsync(off.data(), strong ? t.d_soff : t.d_woff, (size_t)nb * 4,
                                     cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaStreamSynchronize(s));
            int32_t* o = static_cast<int32_t*>(h_dst);
            for (int64_t b = 0; b < nb; ++b) o[b] -= off[(size_t)b];
            return FMM_OK;
        }
        case FMM_EXPORT_STRONG_OFF: return copy(t.d_soff, nb, 4);
        case FMM_EXPORT_STRONG: return copy(t.d_sidx, (int64_t)t.h_counts[0], 4);
        case FMM_EXPORT_WEAK_OFF: return copy(t.d_woff, nb, 4);
        case FMM_EXPORT_WEAK: return copy(t.d_widx, (int64_t)t.h_counts[1], 4);
        case FMM_EXPORT_M2L_ITEMS: return copy(t.d_m2l_items, 4 * (int64_t)t.h_counts[3], 4);
        case FMM_EXPORT_M2L_ROWS: return copy(t.d_m2l_rows, (int64_t)t.h_counts[3], 4);
        case FMM_EXPORT_P2P_ITEMS: return copy(t.d_p2p_items, 4 * (int64_t)t.h_counts[2], 4);
        case FMM_EXPORT_P2P_ROWS: {
            const int64_t m = (int64_t)t.h_counts[2];
            if (count < m) return invalid("host buffer too small");
            std::vector<int32_t> rows((size_t)std::max<long long>(t.p2p_cap, 1));
            unsigned long long nh = 0;
            FMM_CUDA(cudaMemcpyAsync(rows.data(), t.d_p2p_rows, (size_t)t.p2p_cap * 4, cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaMemcpyAsync(&nh, t.d_m2l_rowctr + kM2LItemPairsMax + 1, sizeof(nh), cudaMemcpyDeviceToHost,
                                     s));
            FMM_CUDA(cudaStreamSynchronize(s));
            int32_t* o = static_cast<int32_t*>(h_dst);
            for (int64_t k = 0; k < m; ++k)
                o[k] = (unsigned long long)k < nh ? rows[(size_t)k] : rows[(size_t)(t.p2p_cap - 1 - (k - (int64_t)nh))];
            return FMM_OK;
        }
        case FMM_EXPORT_INST: {
            if (count < 3 * (int64_t)t.ninst) return invalid("host buffer too small");
            int64_t* o = static_cast<int64_t*>(h_dst);
            for (int b = 0; b < t.ninst; ++b) {
                o[3 * b] = t.inst_pt_off[b];
                o[3 * b + 1] = t.inst_box_off[b];
                o[3 * b + 2] = t.inst_levels[b];
            }
            return FMM_OK;
        }
        case FMM_EXPORT_NEAR: {
            if (count < 2 * n) return invalid("host buffer too small");
            if (!t.d_near || t.eval_nbox == 0) return invalid("no evaluation yet");
            // near field per sorted point: in place, or the sum of the leaf's item partials
            double* o = static_cast<double*>(h_dst);
            const bool f32 = t.path == FMM_PATH_FP32;
            const size_t cs = f32 ? 8 : 16;
            const int64_t items = (int64_t)t.h_counts[2];
            std::vector<char> nv(n * cs), pv((size_t)std::max<int64_t>(items, 1) * t.max_leaf * cs);
            std::vector<int2> li(nb);
            FMM_CUDA(cudaMemcpyAsync(nv.data(), t.d_near, nv.size(), cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaMemcpyAsync(pv.data(), t.d_p2p_part, (size_t)items * t.max_leaf * cs,
                                     cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaMemcpyAsync(li.data(), t.d_leaf_items, nb * sizeof(int2), cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaStreamSynchronize(s));
            auto val = [&](const std::vector<char>& v, size_t k, int c) -> double {
                return f32 ? (double)reinterpret_cast<const float*>(v.data())[2 * k + c]
                           : reinterpret_cast<const double*>(v.data())[2 * k + c];
            };
            for (int32_t lf : t.h_leaves) {
                const int2 it = li[lf];
                for (int32_t i = t.h_bstart[lf]; i < t.h_bstart[lf] + t.h_bcount[lf]; ++i) {
                    for (int c = 0; c < 2; ++c) {
                        double acc = 0;
                        if (it.y == 1) {
                            acc = val(nv, i, c);
                        } else {
                            for (int q = 0; q < it.y; ++q)
                                acc += val(pv, (size_t)(it.x + q) * t.max_leaf + (i - t.h_bstart[lf]), c);
                        }
                        o[2 * i + c] = acc;
                    }
                }
            }
            return FMM_OK;
        }
        case FMM_EXPORT_MPOLE:
        case FMM_EXPORT_LOCAL: {
            if (count < 2 * nb * t.p) return invalid("host buffer too small");
            if (t.eval_nbox == 0) return invalid("no evaluation yet");
            const size_t PS = (size_t)t.PS;
            std::vector<double> a64(2 * nb * PS);
            std::vector<float> a32(2 * nb * PS);
            const bool mp = what == FMM_EXPORT_MPOLE;
            if (!mp) {
                // device work on the workspace only; the tree itself is unchanged
                const fmm_status st = complete_folded_locals(const_cast<Tree&>(t), s);
                if (st) return st;
            }
            FMM_CUDA(cudaMemcpyAsync(a64.data(), mp ? t.d_M64 : t.d_L64, a64.size() * 8, cudaMemcpyDeviceToHost, s));
            if (mp && t.path == FMM_PATH_FP32)
                FMM_CUDA(cudaMemcpyAsync(a32.data(), t.d_M32, a32.size() * 4, cudaMemcpyDeviceToHost, s));
            FMM_CUDA(cudaStreamSynchronize(s));
            double* o = static_cast<double*>(h_dst);
            for (int64_t b = 0; b < nb; ++b) {
                const bool leaf32 = mp && t.path == FMM_PATH_FP32 && t.h_child0[b] < 0;
                for (int k = 0; k < t.p; ++k) {
                    const size_t src = 2 * ((size_t)b * PS + k);
                    o[2 * (b * t.p + k)] = leaf32 ? a32[src] : a64[src];
                    o[2 * (b * t.p + k) + 1] = leaf32 ? a32[src + 1] : a64[src + 1];
                }
            }
            return FMM_OK;
        }
    }
    return invalid("unknown export id");
}

}  // extern "C"
