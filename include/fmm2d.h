/*
 * fmm2d.h -- C ABI of the B300 (sm_103a) balanced adaptive 2D FMM library
 * (libfmm2d.so).
 *
 * The library evaluates the 2D harmonic potential in complex form,
 *     Phi(z_i) = sum_{j : z_j != z_i} Gamma_j / (z_i - z_j),   z = x + i y,
 * i.e. the pairwise sum of Sec. 2, eq (2.1), with the exclusion rule of eq (2.2)
 * and the harmonic kernel of Sec. 3.3 (taken with a + sign), by the balanced
 * adaptive FMM of Holm, Engblom, Goude and Holmgren (arXiv:1311.1006):
 *   - a pyramid tree of N_levels full levels whose boxes are split into four
 *     children at exact medians, x first and then y in each half (Sec. 2.2-2.3);
 *   - strong / weak coupling lists from the theta-criterion R + theta r <= theta d
 *     (Sec. 2.1, eq 2.3);
 *   - P2M, M2M, M2L, L2L, L2P and the P2P near-field sum (Sec. 2.1, Fig 2.2),
 *     all as CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 *   - Device pointers are CUDA device addresses on the current device; host
 *     pointers are ordinary host memory.  The caller owns every buffer it passes;
 *     the library only reads/writes them, asynchronously, on the given stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls return once the work is enqueued, except where stated
 *     (tree builds synchronise the stream once to read a status word).
 *   - Points are N x 2 float64, row-major (x0, y0, x1, y1, ...).  Complex
 *     arrays are interleaved (re, im): float64 pairs, or float32 pairs where a
 *     call says "complex64".
 *   - Outputs are in the caller's input order.  Sources and evaluation points
 *     are the same point set (eq 2.1).  Real strengths: pass im = 0.
 *   - Coincident points (eq 2.2): a pair with z_j == z_i adds nothing.  The P2P
 *     kernels test this through |z_i - z_j|^2 instead of exact equality, so a
 *     pair closer than the resolution of that square also adds nothing: below
 *     about 1e-19 on FMM_PATH_FP32 (|d|^2 under the smallest normal float) and
 *     about 1e-154 on FMM_PATH_FP64 (|d|^2 under the smallest normal double).
 *   - Errors are returned as fmm_status codes; nothing crosses the ABI as an
 *     exception.  fmm_last_error() gives a thread-local detail string.  An
 *     asynchronous CUDA error from earlier work is reported by the next call.
 *   - Two precision paths (fmm_params.path):
 *       FMM_PATH_FP32 (mixed): P2P, M2L, P2M and L2P compute in FP32 with FP32
 *         accumulation; M2M and L2L shifts and the accumulation of expansions
 *         across levels are FP64; output complex64.
 *       FMM_PATH_FP64: every pass in FP64; output complex128.
 *   - Thread safety: a tree may be used by one host thread at a time.
 */
#ifndef FMM2D_H
#define FMM2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID_ARG = 1, /* a size, parameter or pointer is out of range */
    FMM_ERR_CUDA = 2,        /* a CUDA runtime call or kernel failed */
    FMM_ERR_OOM = 3,         /* device or host allocation failed */
    FMM_ERR_TIMEOUT = 4,     /* a bounded device wait ran out (status word) */
    FMM_ERR_NONFINITE = 5    /* NaN / Inf in the point coordinates */
} fmm_status;

typedef enum { FMM_PATH_FP32 = 0, FMM_PATH_FP64 = 1 } fmm_path;

/* fmm_params.flags */
enum {
    FMM_FLAG_NO_GRAPH = 1, /* launch the kernels one by one (the default; overrides FMM_FLAG_GRAPH) */
    FMM_FLAG_SERIAL = 2,   /* run P2P on the caller's stream after the far field (no overlap) */
    FMM_FLAG_TIMING = 4,   /* record per-phase CUDA events; read them with fmm_phase_times */
    FMM_FLAG_GRAPH = 8,    /* capture the evaluation once per (strengths, output, stream) and replay the
                              CUDA graph; fewer host launches, but on B300 the replay overlaps P2P with
                              the far field less well than direct launches on prioritised streams */
    FMM_FLAG_PERSISTENT = 16 /* FMM_PATH_FP32 only: fmm_eval / fmm_eval_batched run the whole evaluation of
                              the tree (every instance of a forest) as ONE persistent kernel whose CTAs take
                              (stage, box range) units from a device work queue in ticket order and wait,
                              bounded, for the units each stage depends on; M2L runs on the CUDA cores.
                              With FMM_FLAG_GRAPH the one launch is captured and replayed.  The
                              logarithmic kernel, the adjoint and separate evaluation points ignore it.
                              A wait that ran out is reported by fmm_eval_status. */
};

/* Maximum expansion order accepted (p terms, coefficients k = 0..p-1). */
#define FMM_P_MAX 32

typedef struct {
    int p;        /* expansion terms, 1 <= p <= FMM_P_MAX (Sec. 2.1, "p terms") */
    double theta; /* separation parameter of eq (2.3), 0 < theta < 1 */
    int nlevels;  /* N_levels >= 1 with 4^(N_levels-1) <= N (no empty leaf);
                     0 = fmm_default_nlevels(N, p, path) */
    int path;     /* fmm_path */
    int flags;    /* FMM_FLAG_* */
} fmm_params;

/* Opaque, device-resident tree + workspace, owned by the library. */
typedef struct fmm_tree fmm_tree;

/* Build the pyramid tree and the coupling lists of one point set (Sec. 2.1-2.3).
 *   d_xy   : device, N x 2 float64 points; read during the call only.
 *   n      : N >= 1 (and < 2^31).
 *   prm    : host, parameters (copied).
 *   out    : host, receives the new tree (NULL on failure).
 * Synchronises `stream` once to check the device status word.
 * Errors: INVALID_ARG (bad n / prm), NONFINITE (NaN or Inf coordinate), OOM, CUDA. */
fmm_status fmm_build_tree(const double* d_xy, int64_t n, const fmm_params* prm, void* stream, fmm_tree** out);

/* Rebuild an existing tree in place for new coordinates of the same N points
 * (the paper rebuilds the partition at every time step, Sec. 3.1), optionally
 * with new parameters (prm may be NULL = keep).  Buffers are reused and grown
 * when needed.  Same errors as fmm_build_tree. */
fmm_status fmm_tree_rebuild(fmm_tree* t, const double* d_xy, const fmm_params* prm, void* stream);

/* Batched build: B independent instances in one forest (one launch per phase
 * covers every instance).  Instance b owns points h_offsets[b] .. h_offsets[b+1]-1
 * of d_xy (h_offsets: host, B+1 entries, h_offsets[0] = 0).  h_nlevels (host, B
 * entries) gives N_levels per instance, or NULL to choose each instance's
 * N_levels with fmm_default_nlevels.  No coupling crosses instances. */
fmm_status fmm_build_tree_batched(const double* d_xy, const int64_t* h_offsets, int B, const fmm_params* prm,
                                  const int* h_nlevels, void* stream, fmm_tree** out);

/* Evaluate Phi at every point (Sec. 2.1: P2M, M2M, M2L, L2L, L2P, P2P).
 *   d_gamma : device, N complex strengths (complex128), input order.
 *   d_phi   : device, N complex outputs, input order: complex64 for
 *             FMM_PATH_FP32, complex128 for FMM_PATH_FP64.
 * Works on single and batched trees.  Errors: INVALID_ARG (NULL), CUDA. */
fmm_status fmm_eval(fmm_tree* t, const double* d_gamma, void* d_phi, void* stream);

/* Same as fmm_eval; rejects a tree that was not built by fmm_build_tree_batched. */
fmm_status fmm_eval_batched(fmm_tree* t, const double* d_gamma, void* d_phi, void* stream);

/* One time step: fmm_tree_rebuild(t, d_xy, NULL, stream) followed by
 * fmm_eval(t, d_gamma, d_phi, stream), same arguments and the same result bit
 * for bit, in one call that overlaps the two: the strength gather and the
 * upward pass (P2M, M2M), which need the tree but not the coupling lists, run
 * on the library's far-field stream while the lists are built.  Once an
 * earlier build has sized the list and item capacities, the evaluation is
 * queued on the device behind the list passes and the host checks the
 * build's counters while it runs; the call returns when that check is done
 * (the evaluation may still be running on `stream`).  A build that needs
 * larger capacities (or met a non-finite coordinate or a long run of equal
 * coordinates) is done again in the checked order, into the same d_phi.
 * Parameters stay as the tree has them (change them with fmm_tree_rebuild).
 * A batched tree, or a tree with FMM_FLAG_SERIAL, FMM_FLAG_TIMING,
 * FMM_FLAG_GRAPH or FMM_FLAG_PERSISTENT, runs the two calls in sequence.
 * Errors: INVALID_ARG (NULL, a tree built with separate evaluation points),
 * CUDA, OOM, TIMEOUT, NONFINITE as the two calls. */
fmm_status fmm_step(fmm_tree* t, const double* d_xy, const double* d_gamma, void* d_phi, void* stream);

/* Self-test of the library's bounded device waits (failure detection without
 * a GPU fault): runs one of them on something that never happens -- which = 0:
 * the decoupled look-back of the list build, partitions and sorts on a
 * predecessor tile that never publishes; which = 1: the tensor-core M2L's
 * mbarrier wait on a barrier nothing arrives at; which = 2: the persistent
 * evaluation's wait for a stage's dependencies on a unit that never completes
 * -- with a short limit (4096 tries).  The expected result is FMM_ERR_TIMEOUT,
 * returned from the device's status word; the context stays usable.
 * Errors: INVALID_ARG (which), CUDA. */
fmm_status fmm_selftest_bounded_wait(int which, void* stream);

/* Status of the last evaluation's bounded device waits (the tensor-core
 * M2L's mbarrier waits, the persistent evaluation's queue waits): synchronises
 * `stream` and returns FMM_ERR_TIMEOUT if one of them ran out (its results are
 * then incomplete), else FMM_OK.  Call it after the evaluation and before the
 * next build or rebuild of the tree, which clears the status word.
 * Errors: INVALID_ARG (NULL), CUDA, TIMEOUT. */
fmm_status fmm_eval_status(fmm_tree* t, void* stream);

/* Diagnostic: d_out[i] = the FP64 P2P's reciprocal of d_x[i] (n doubles,
 * device buffers): the hardware's approximate reciprocal refined by two
 * Newton-Raphson steps; 0 for inputs below the smallest normal double.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
fmm_status fmm_selftest_rcp64(const double* d_x, double* d_out, int64_t n, void* stream);

/* Logarithmic potential (Sec. 3.3 of the paper, the kernel it uses for
 * isopotential plots):
 *     Phi_i = sum_{j: z_j != z_i} Gamma_j ln|z_i - z_j|,
 * complex strengths acting on the real kernel (the real and imaginary parts of
 * Gamma give the real and imaginary parts of Phi).  Same tree, lists, expansion
 * order and precision path as fmm_eval; the log multipole is the integral of
 * the harmonic one (a_0 log(z - c) + sum_{k>=1} a_k/(z - c)^k, locals of degree
 * p), so the far field runs the harmonic passes twice (one real-strength set
 * per part of Gamma) plus the constant term of each local expansion, and P2P
 * takes one logarithm per pair.  Arguments as fmm_eval (d_gamma: n complex128,
 * caller's order; d_phi: n complex64 on the FP32 path, complex128 on FP64).
 * fmm_eval_targets_log is the same at the evaluation points of a tree built
 * by fmm_build_tree_targets (as fmm_eval_targets).  Errors: INVALID_ARG, CUDA,
 * OOM. */
fmm_status fmm_eval_log(fmm_tree* t, const double* d_gamma, void* d_phi, void* stream);
fmm_status fmm_eval_targets_log(fmm_tree* t, const double* d_gamma, void* d_phi, void* stream);

/* Adjoint of fmm_eval with the tree frozen.  For the real loss
 *     L = sum_i w_i Re Phi_i + v_i Im Phi_i,    d_gphi[i] = w_i + i v_i (complex128),
 * writes (torch convention: d/dRe + i d/dIm)
 *     d_ggamma[k] = dL/dRe Gamma_k + i dL/dIm Gamma_k = -conj(Psi_k)   (complex128)
 *     d_gxy[k]    = (dL/dx_k, dL/dy_k) = (Re D_k, -Im D_k)             (N x 2 float64)
 * with c = conj(gphi), Psi(z) = sum_i c_i/(z - z_i) (a second FMM over the same
 * tree), D_k = c_k Phi'(z_k) - Gamma_k Psi'(z_k).  Either output may be NULL.
 * Uses the tree's precision path.  Errors: INVALID_ARG, CUDA. */
fmm_status fmm_eval_backward(fmm_tree* t, const double* d_gamma, const double* d_gphi, double* d_ggamma,
                             double* d_gxy, void* stream);

/* Separate evaluation points (eq 2.2): Phi(y_i) = sum_{j: x_j != y_i} Gamma_j / (y_i - x_j)
 * at n_tgt points y (d_tgt_xy, n_tgt x 2 float64, device) for n_src sources x
 * (d_src_xy, n_src x 2 float64, device).  The tree is built over the sources and
 * the evaluation points together, the evaluation points carrying zero strength
 * (they change no expansion; the P2P pass skips coincident points, which is
 * x_j != y_i), so the balanced splits see all n_src + n_tgt points.
 * fmm_eval_targets: d_gamma = n_src complex128 source strengths, d_phi = n_tgt
 * complex values (complex64 on the FP32 path, complex128 on FP64).  The library
 * keeps copies of the points and strengths in its own workspace.  N_levels is
 * chosen for n_src + n_tgt points.  Errors: INVALID_ARG (NULL, n < 1, a tree not
 * built with fmm_build_tree_targets), CUDA, OOM. */
fmm_status fmm_build_tree_targets(const double* d_src_xy, int64_t n_src, const double* d_tgt_xy, int64_t n_tgt,
                                  const fmm_params* params, void* stream, fmm_tree** out);
fmm_status fmm_tree_rebuild_targets(fmm_tree* t, const double* d_src_xy, const double* d_tgt_xy,
                                    const fmm_params* params, void* stream);
fmm_status fmm_eval_targets(fmm_tree* t, const double* d_gamma, void* d_phi, void* stream);

/* One step of the autotuner (Sec. 4.2, Algorithm 4 "AT3b": a directed walk
 * with cost estimation and a user cap on the tuning cost).  Call after every
 * evaluation with its time; *inout receives the parameters to use next
 * (nlevels; with fmm_autotune_theta also theta and p, else theta is kept and p
 * untouched).  The caller rebuilds the tree with them (fmm_tree_rebuild).
 * Host-only; no device work. */
fmm_status fmm_autotune_step(fmm_tree* t, double last_time_s, fmm_params* inout);

/* Tune theta as well (the theta moves of Algorithms 2-4, Sec. 4.2): moves of
 * 0.01 x Fibonacci steps alternating with N_levels moves; a rejected move
 * reverses direction and takes the next step of the sequence.  p follows
 * theta through the tolerance: p = fmm_p_for_tolerance(tol, theta).  theta is
 * kept in [theta_min, theta_max] and where p <= FMM_P_MAX.
 * Errors: INVALID_ARG (0 < tol < 1, 0 < theta_min <= theta_max < 1 and
 * p(tol, theta_min) <= FMM_P_MAX required). */
fmm_status fmm_autotune_theta(fmm_tree* t, double tol, double theta_min, double theta_max);

/* Expansion terms for relative tolerance tol at separation theta (Sec. 4.1,
 * p ~ log TOL / log theta): ceil(0.9 ln(tol) / ln(theta)); never below the
 * paper's Table 4.1 and at most one above it.  -1 for arguments outside (0,1). */
int fmm_p_for_tolerance(double tol, double theta);

/* Configure the autotuner: cap = maximum relative tuning cost (e.g. 0.1),
 * window = number of evaluations whose minimum time is used per decision
 * (noise filter, Sec. 4.2.1), period = evaluations between N_levels moves. */
fmm_status fmm_autotune_config(fmm_tree* t, double cap, int window, int period);

/* Standalone N_levels autotuner with the same AT3b logic, for callers that
 * manage trees themselves (and for host-only tests).  nlevels = starting
 * N_levels, max_levels = largest allowed (4^(max_levels-1) <= N).
 * fmm_autotuner_step takes the last evaluation time and writes the N_levels
 * to use next.  fmm_autotuner_stats writes up to 6 values: accepted N_levels,
 * steps, rejected moves, time lost to rejected moves (s), accumulated time of
 * accepted evaluations (s), N_levels on trial (0 = none). */
typedef struct fmm_autotuner fmm_autotuner;
fmm_status fmm_autotuner_create(int nlevels, int max_levels, double cap, int window, int period,
                                fmm_autotuner** out);
fmm_status fmm_autotuner_step(fmm_autotuner* a, double time_s, int* nlevels_out);
/* Enable theta moves on a standalone tuner (as fmm_autotune_theta), starting at theta. */
fmm_status fmm_autotuner_theta(fmm_autotuner* a, double theta, double tol, double theta_min, double theta_max);
/* As fmm_autotuner_step, also writing theta and p to use next (p = -1 without theta moves). */
fmm_status fmm_autotuner_step_params(fmm_autotuner* a, double time_s, int* nlevels_out, double* theta_out,
                                     int* p_out);
/* Up to 8 values: the 6 above, then the accepted theta and the theta on trial (0 = none). */
fmm_status fmm_autotuner_stats(const fmm_autotuner* a, double* out, int nout);
void fmm_autotuner_destroy(fmm_autotuner* a);

/* Cost-model seed of N_levels (Sec. 2.3, eqs 2.4-2.5; the starting point of
 * the autotuner, Sec. 4.2).  With N_f = 4^(N_levels-1) leaves the model counts
 *     C_P2P = N^2/(2 N_f) * pi((1+theta)/theta)^2,
 *     C_M2L = (3 N_f/2) p^2 * pi((1+theta)/theta)^2,
 * and with unit costs alpha (seconds per unit of C_P2P) and beta (per unit of
 * C_M2L) the time alpha C_P2P + beta C_M2L is smallest at
 *     N_f* = (N/p) sqrt(alpha / (3 beta)).
 * fmm_seed_nlevels returns the N_levels in [1, largest with 4^(N_levels-1) <= n]
 * whose N_f is closest to N_f* on a log scale (0 for n < 1, p < 1 or
 * alpha, beta <= 0).  Host-only. */
int fmm_seed_nlevels(int64_t n, int p, double alpha, double beta);

/* N_levels the library picks for n points at expansion order p when
 * fmm_params.nlevels == 0: fmm_seed_nlevels with the library's unit costs
 * for `path` (fmm_cost_model_get). */
int fmm_default_nlevels(int64_t n, int p, int path);

/* The library's unit costs (alpha, beta) of the cost model above, one pair
 * per precision path, shared by the whole process.  Built in: values measured
 * on B300 (1e6-point cluster set, p = 17, theta = 0.5, N_levels = 9, P2P and
 * M2L each timed alone).  fmm_cost_model_calibrate replaces the pair of the
 * tree's path with the unit costs measured in the tree's last evaluation:
 * alpha = P2P time / C_P2P, beta = M2L time / C_M2L (model counts summed over
 * the instances of a batched tree).  That evaluation must have been made with
 * FMM_FLAG_TIMING (with FMM_FLAG_SERIAL too, P2P and M2L are timed alone and
 * the unit costs do not include their overlap) on a tree with N_levels >= 3.
 * The measured pair is written to *alpha_out, *beta_out (either may be NULL).
 * Errors: INVALID_ARG (no timed evaluation, no M2L work, bad path or values),
 * CUDA.  fmm_cost_model_set sets a pair directly (alpha, beta > 0, finite). */
fmm_status fmm_cost_model_calibrate(fmm_tree* t, double* alpha_out, double* beta_out);
fmm_status fmm_cost_model_get(int path, double* alpha, double* beta);
fmm_status fmm_cost_model_set(int path, double alpha, double beta);

/* Per-phase device times (milliseconds) of the last evaluation made with
 * FMM_FLAG_TIMING: out[0] gather, [1] P2M+M2M, [2] M2L, [3] L2L, [4] P2P,
 * [5] L2P+combine, [6] whole evaluation.  Synchronises on the recorded events. */
fmm_status fmm_phase_times(fmm_tree* t, double* out, int nout);

/* Tree facts (host struct). */
typedef struct {
    int64_t n;               /* points */
    int ninst;               /* instances (1 unless batched) */
    int nlevels_max;         /* largest N_levels over instances */
    int p, path;
    double theta;
    int64_t nboxes;          /* boxes over all levels and instances */
    int64_t nleaves;
    int64_t n_strong;        /* strong-list entries over all levels */
    int64_t n_weak;          /* weak-list entries = M2L pairs over all levels */
    int64_t n_strong_leaf;   /* P2P leaf pairs */
    int64_t p2p_pairs;       /* P2P point pairs: sum over leaves of n_leaf * near points */
    int64_t p2p_items;       /* P2P work items (a leaf with a long strong list is split) */
    int64_t m2l_items;       /* M2L work items */
    int autotune_nlevels;    /* N_levels the autotuner has accepted so far */
    int launches_build;      /* kernels one build / rebuild launches */
    int launches_eval;       /* kernels one evaluation launches */
    double autotune_theta;   /* theta the autotuner has accepted (the tree's theta without theta moves) */
} fmm_tree_info;

/* Fills *out; the pair counts are summed on the device (synchronises). */
fmm_status fmm_get_tree_info(const fmm_tree* t, fmm_tree_info* out);

/* Copy one of the tree's device arrays to host memory (tests, diagnostics).
 * `count` is the number of ELEMENTS the host buffer holds; the call fails
 * with INVALID_ARG when it is too small.  Synchronises `stream`. */
typedef enum {
    FMM_EXPORT_PERM = 0,      /* int32[n]     sorted position -> input index */
    FMM_EXPORT_BSTART = 1,    /* int32[nbox]  first sorted position of each box */
    FMM_EXPORT_BCOUNT = 2,    /* int32[nbox]  points in each box */
    FMM_EXPORT_CENTER = 3,    /* float64[2*nbox] */
    FMM_EXPORT_RADIUS = 4,    /* float64[nbox] */
    FMM_EXPORT_NSTRONG = 5,   /* int32[nbox]      strong-list length of each box */
    FMM_EXPORT_STRONG = 6,    /* int32[n_strong]  strong-list entries (CSR; box b: STRONG_OFF[b] ..) */
    FMM_EXPORT_NWEAK = 7,     /* int32[nbox] */
    FMM_EXPORT_WEAK = 8,      /* int32[n_weak] */
    FMM_EXPORT_MPOLE = 9,     /* float64[2*nbox*p]: multipole coefficients a_k / rho^k (rho = scale radius) */
    FMM_EXPORT_LOCAL = 10,    /* float64[2*nbox*p]: local coefficients b_l * rho^l */
    FMM_EXPORT_NEAR = 11,     /* float64[2*n]: P2P part of the last evaluation, sorted order */
    FMM_EXPORT_INST = 12,     /* int64[3*ninst]: point offset, box offset, N_levels per instance */
    FMM_EXPORT_RHO = 13,      /* float64[nbox]: scale radius rho of each box */
    FMM_EXPORT_STRONG_OFF = 14, /* int32[nbox]  first entry of each strong list */
    FMM_EXPORT_WEAK_OFF = 15,   /* int32[nbox] */
    FMM_EXPORT_M2L_ITEMS = 16,  /* int32[4*m2l_items]: M2L work items (box, list begin, list end, first item of
                                   the box or -1), a box's items consecutive */
    FMM_EXPORT_M2L_ROWS = 17,   /* int32[m2l_items]: the order in which the M2L kernels take the items (row ->
                                   item): full items first, then each box's shorter last item by decreasing length */
    FMM_EXPORT_P2P_ITEMS = 18,  /* int32[4*p2p_items]: P2P work items (leaf, strong-list begin, end, first item of
                                   the leaf or -1), a leaf's items consecutive */
    FMM_EXPORT_P2P_ROWS = 19    /* int32[p2p_items]: the order in which the P2P kernels take the items (ticket ->
                                   item): the full items of split leaves first, then every leaf's last or only item */
} fmm_export_what;

fmm_status fmm_tree_export(const fmm_tree* t, int what, void* h_dst, int64_t count, void* stream);

void fmm_tree_destroy(fmm_tree* t);

/* Exact pairwise sum Phi(z_i) = sum_{z_j != z_i} Gamma_j / (z_i - z_j) for at
 * most 16384 points, in FP64, that ALLOCATES NO DEVICE MEMORY.  The paper has no
 * counterpart: it is an addition for callers that cannot allocate — code inside
 * a host application that owns every device allocation (a fixed pool handed out
 * by a framework), or latency-critical loops where cudaMalloc/cudaFree, which
 * can synchronise the device, are not allowed.
 *   d_xy    : device, n x 2 float64 points;  d_gamma : device, n complex128
 *   d_phi   : device, n complex128 outputs (input order)
 * Scratch: a fixed 2 MiB __device__ array inside the library, resident on every
 * GPU that loads it until the process exits.  Every call looks up that array's
 * device address on the current device (no allocation, no synchronisation; the
 * address stays right after cudaDeviceReset); the first call on a device may
 * load the library's device code, so make it before any stream capture.  All
 * calls share the array, so calls that run at the same
 * time on one GPU (unordered streams) race and give wrong results; calls
 * ordered on one stream are safe, and nothing needs clearing between them.
 * Errors: INVALID_ARG (NULL pointer, n < 1 or n > 16384), CUDA. */
fmm_status fmm_direct_eval_noalloc(const double* d_xy, const double* d_gamma, int64_t n, double* d_phi,
                                   void* stream);

const char* fmm_status_string(fmm_status s);
const char* fmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FMM2D_H */
