// Internal declarations of the B300 FMM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fmm2d.h"

namespace fmm {

// ------------------------------------------------ programmatic dependent launch
// The build is a chain of short kernels on one stream.  A kernel launched by
// launch_dep(true, ...) is scheduled as the kernel before it in the stream
// finishes (its launch overlaps the other's last CTAs); pdl_wait(), its first
// statement, waits until every prerequisite grid has completed and its memory
// writes are visible, so no memory access of the kernel precedes that point.
// No kernel triggers its dependents early (griddepcontrol.launch_dependents):
// that measured ~8 us more per step but keeps grids' CTAs waiting on the SMs
// ahead of time.  Without the launch attribute the wait does nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... K, typename... A>
inline cudaError_t launch_dep(bool dep, void (*k)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = dep ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

// ------------------------------------------------------------------ status
// Bits of the device status word (atomicOr from kernels, read after a build).
enum : unsigned {
    ST_NONFINITE = 1u,        // NaN/Inf coordinate seen by the key kernel
    ST_STRONG_OVERFLOW = 2u,  // a strong list exceeded its fixed capacity
    ST_WEAK_OVERFLOW = 4u,    // a weak list exceeded its fixed capacity
    ST_TIMEOUT = 8u,          // a bounded wait gave up
    ST_INTERNAL = 16u,        // an index check in a scatter failed (a bug, reported not written)
    ST_ITEM_OVERFLOW = 32u,   // a work-item array exceeded its capacity
    ST_SORT_RUN = 64u         // the short coordinate sort met a run of equal high halves it does not resolve
};

// P2P lane layout for leaves of at most max_leaf points: lt target lanes x
// 32/lt source slices, tpl targets per lane.
struct P2PLayout {
    int tpl, lt;
};
inline P2PLayout p2p_layout(int max_leaf) {
    if (max_leaf <= 4) return {2, 2};
    if (max_leaf <= 8) return {4, 2};
    if (max_leaf <= 16) return {8, 2};
    if (max_leaf <= 32) return {8, 4};
    if (max_leaf <= 64) return {8, 8};
    return {8, 16};
}
// FP32 path: lanes take PAIRS of source slots (packed f32x2 arithmetic), so a
// step covers 2 * 32/lt slots.
inline P2PLayout p2p_pair_layout(int max_leaf) {
    if (max_leaf <= 8) return {2, 4};
    if (max_leaf <= 16) return {4, 4};
    if (max_leaf <= 32) return {4, 8};
    if (max_leaf <= 64) return {4, 16};
    return {8, 16};
}
// Slots per leaf: max_leaf rounded up to whole source steps of both layouts
// (the pair layout's step is a multiple of the scalar layout's).
inline int leaf_capacity(int max_leaf) {
    const int step = 2 * (32 / p2p_pair_layout(max_leaf).lt);
    return (max_leaf + step - 1) / step * step;
}

// Work-item sizes: P2P items hold about this many source points; M2L items at
// most this many weak pairs.
constexpr int kP2PItemSources = 4096;  // measured: 4096 beats 2048 (+0.3 %) and 8192 (+3 %) on the 1e6-point step
// Source points per P2P work item: kP2PItemSources from half a million points up; smaller trees take
// proportionally smaller items (at least 256 sources), so that their few leaves still give the GPU enough
// warps (the split leaves' partial sums are added in item order, as for the long lists of large trees).
inline int p2p_item_sources(int64_t n) {
    const int64_t big = int64_t(1) << 19;
    if (n >= big) return kP2PItemSources;
    return (int)std::max<int64_t>(256, (int64_t)kP2PItemSources * n / big);
}
constexpr int kMaxLevels = 16;
constexpr int kSubMax = 4096;  // largest box whose remaining splits one CTA performs in shared memory
constexpr int kM2LItemPairsMax = 256;  // bound of m2l_item_pairs (counters of the M2L row order)
constexpr int kM2LTcRows = 128;  // work items (MMA rows) per CTA of the tensor-core M2L

// Partition tile: 256 threads x 8 consecutive positions.
constexpr int kPartThreads = 256;
constexpr int kPartItems = 4;  // measured: 4 beats 8 (rebuild 1.062 -> 1.034 ms), 2, 3 and 6; 128 threads x 4 slower
constexpr int kPartTile = kPartThreads * kPartItems;

// Radix sort tile: 256 threads x 8 rounds.
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;

// Segment table of one partition stage: segment k covers sorted positions
// [start[k], start[k+1]) and its first nzero[k] positions (by the list being
// split) keep flag 0.
struct SegTable {
    int K = 0;
    int32_t* d_start = nullptr;    // K+1 entries, start[K] = n
    int32_t* d_nzero = nullptr;    // K entries
    int32_t* d_obefore = nullptr;  // K entries: flag-1 positions in segments before k
};

struct LevelList {
    int count = 0;
    int32_t* d_ids = nullptr;  // global box ids
};

// --------------------------------------------------------------- the tree
struct Tree {
    // separate evaluation points (eq 2.2): the tree holds n_src sources followed by n_tgt
    // evaluation points of zero strength (n_src == 0: sources are the evaluation points)
    int64_t n_src = 0, n_tgt = 0;
    double* d_xy_all = nullptr;   // sources then evaluation points
    double* d_gam_all = nullptr;  // source strengths then zeros
    void* d_phi_all = nullptr;    // potentials of all points (path precision)
    int phi_all_path = -1;

    // parameters
    int p = 17, P = 17, PS = 18, path = FMM_PATH_FP32, flags = 0;
    double theta = 0.5;
    bool batched = false;
    // coordinate sort: false = the high 32 key bits by radix passes, then the short runs of equal high halves
    // in place; true (set for good once a build met a longer run) = all 64 bits by radix passes
    bool sort_full = false;

    // shape
    int64_t n = 0;
    int ninst = 1;
    std::vector<int64_t> inst_pt_off;   // ninst+1
    std::vector<int> inst_levels;       // ninst
    std::vector<int64_t> inst_box_off;  // ninst+1
    int Lmax = 1;
    int64_t nbox = 0, nleaf = 0;
    std::vector<int64_t> shape_key;     // (inst sizes, levels) the tables were built for

    // host copies of the shape tables
    std::vector<int32_t> h_bstart, h_bcount, h_parent, h_child0, h_inst;
    std::vector<std::vector<int32_t>> h_level_boxes;  // per level: boxes present
    std::vector<int32_t> h_leaves;

    // device shape tables
    int32_t *d_bstart = nullptr, *d_bcount = nullptr, *d_parent = nullptr, *d_child0 = nullptr,
            *d_inst = nullptr;
    // per box: for the leaves of the deepest level (N_levels >= 3) their parent, else -1.  On the FP32 path
    // these leaves get no L2L: L2P evaluates the parent's local expansion at the point and adds the
    // leaf's own M2L sum (the shift of a truncated local is an exact re-expansion of the same polynomial)
    int32_t* d_fold_par = nullptr;
    std::vector<LevelList> level_boxes;    // per level l: all boxes on level l
    std::vector<LevelList> level_parents;  // per level l: boxes on level l that have children
    LevelList leaves;
    std::vector<SegTable> seg_x, seg_y;    // per level l < Lmax-1
    int64_t* d_inst_ptoff = nullptr;       // ninst+1
    int32_t* d_inst_levels = nullptr;      // ninst
    int l0 = 0;                            // first level split inside one CTA per box
    int64_t* d_inst_boxoff = nullptr;      // ninst+1 (root box id of each instance)
    int32_t* d_leaf_start = nullptr;       // nleaf+1: first sorted position of each leaf
    // leaf slot layout of the P2P operands: leaf q owns slots [q*leaf_cap, (q+1)*leaf_cap);
    // its points fill the first bcount slots, the rest (and one extra block after the
    // last leaf) are padding with zero strength
    int leaf_cap = 16;
    int32_t* d_pslot = nullptr;            // per box: first slot of a leaf, -1 otherwise

    // build scratch
    uint64_t* d_keys[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t* d_vals[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t *d_X2 = nullptr, *d_Y2 = nullptr;
    uint8_t *d_sideX = nullptr, *d_sideY = nullptr;
    int32_t* d_loc = nullptr;  // input index -> local id inside a subtree CTA
    unsigned long long* d_part_stat = nullptr;  // partition: tile status words + tile ticket
    int32_t *d_sort_hist = nullptr, *d_sort_tot = nullptr, *d_sort_off = nullptr;
    unsigned* d_sort_os = nullptr;  // onesweep sort: global digit counts, tickets, tile status words
    int64_t segs_cap = 0;

    // tree data
    int32_t* d_perm = nullptr;     // sorted position -> input index
    int32_t* d_leaf_of = nullptr;  // sorted position -> leaf box id
    double2* d_pts = nullptr;      // sorted FP64 points
    float4* d_pos4 = nullptr;      // sorted (x_hi, y_hi, x_lo, y_lo) relative to the instance origin
    void* d_posp = nullptr;        // slot layout, 16 B per slot: FP64 points, or on the FP32 path the
                                   // pair-interleaved hi/lo coordinates (see k_finalize)
    int32_t* d_slot_of = nullptr;  // sorted position -> slot
    // separate evaluation points: per leaf the number of SOURCES; a leaf's slot block holds its sources first
    // and its evaluation points after them, so P2P takes sources [0, nsrc) and targets [nsrc, count) of a block
    int32_t* d_nsrc = nullptr;
    int64_t slot_alloc = 0;        // slots d_posp was allocated for
    double2* d_center = nullptr;   // per box
    double* d_radius = nullptr;    // per box (half bbox diagonal)
    double* d_rho = nullptr;       // per box scale radius = (double)(float)radius
    float4* d_chl = nullptr;       // per box centre hi/lo relative to the instance origin
    float* d_rho32 = nullptr;      // per box (float)rho
    float* d_rad32 = nullptr;      // per box (float)radius, for the FP32 pre-test of eq (2.3)
    // coupling lists in CSR form: box b's strong list is sidx[soff[b] .. soff[b]+ns[b])
    int32_t *d_soff = nullptr, *d_ns = nullptr, *d_sidx = nullptr;
    int2* d_srng = nullptr;        // leaves: (first slot, count) of each strong entry, parallel to sidx
    int32_t* d_sowner = nullptr;   // box of each strong entry, parallel to sidx
    unsigned long long* d_ltstat = nullptr;  // list build: tile status words (strong, weak) + tile ticket
    unsigned long long* d_lvl_base = nullptr;  // [0,16) strong / [16,32) weak level offsets, [32,36) sizes needed
    long long cand_cap = 0;
    int32_t *d_woff = nullptr, *d_nw = nullptr, *d_widx = nullptr;
    long long scap_tot = 0, wcap_tot = 0;
    // work items (see k_items)
    int4* d_p2p_items = nullptr;
    // P2P row order (ticket -> item): the full items of split leaves first (rows from the front), then every
    // leaf's last or only item (rows from the back of the capacity), so the long items do not make the tail
    int32_t* d_p2p_rows = nullptr;
    int4* d_m2l_items = nullptr;
    int2* d_leaf_items = nullptr;  // per box: first P2P item, item count (leaves)
    int2* d_box_m2l = nullptr;     // per box: first M2L item, item count
    // row order of the M2L kernels: every full item (m2l_item_pairs() pairs) first, then the boxes' shorter
    // last items by decreasing length, so that threads stepping through their items in lockstep (a warp, or
    // the CTA of the tensor-core M2L) have about the same number of pairs
    int32_t* d_m2l_rows = nullptr;              // m2l_cap: row -> item
    int2* d_box_tail = nullptr;                 // per box: (length of its short last item or 0, rank among equals)
    unsigned long long* d_m2l_rowctr = nullptr;  // [kM2LItemPairsMax + 1]: short items per length, then full items
    long long p2p_cap = 0, m2l_cap = 0;
    // work items the P2P / M2L launch grids cover: the last build's counts plus
    // slack, re-derived (and the evaluation graph re-captured) when a build's
    // counts leave [grid/2.5, grid]
    long long grid_p2p_items = 0, grid_m2l_items = 0;
    int max_leaf = 1;
    int num_sms = 148;              // largest leaf (points): row stride of the P2P partial sums
    // device words: [0] status bits, then 64-bit counters:
    // [1] strong entries, [2] weak entries, [3] P2P items, [4] M2L items, [5..6] diagnostics
    unsigned* d_status = nullptr;
    unsigned long long h_counts[4] = {0, 0, 0, 0};  // strong, weak, P2P items, M2L items

    // evaluation workspace
    void* d_gam = nullptr;     // sorted strengths (float2 or double2), 2 sets for backward
    void* d_gamp = nullptr;    // strengths in the leaf slot layout (forward set)
    int64_t eval_slots = 0;
    void* d_gamp2 = nullptr;   // adjoint, FP32 path: the second strength set c in the slot layout
    int64_t gamp2_slots = 0;
    void* d_near = nullptr;    // P2P output(s), sorted order
    void* d_p2p_part = nullptr;  // partial P2P sums of split leaves (item x max_leaf)
    void* d_m2l_part = nullptr;  // partial M2L sums of split boxes (item x PS)
    long long part_p2p_cap = 0, part_m2l_cap = 0;
    bool parts_stale = true;  // partial-sum buffers must be (re)allocated before use
    double2* d_M64 = nullptr;  // multipoles, scaled
    float2* d_M32 = nullptr;
    void* d_Lm2l = nullptr;    // M2L sums per box
    double2* d_L64 = nullptr;  // locals after L2L, scaled
    float2* d_L32 = nullptr;
    size_t eval_nbox = 0, eval_n = 0;
    int eval_ts = 0;
    int eval_PS = 0, eval_path = -1, eval_sets = 0;
    unsigned eval_gen = 0;  // bumped whenever alloc_eval reallocates (captured graphs hold the old pointers)

    // streams / events
    cudaStream_t s_aux = nullptr;  // P2P (lowest priority)
    cudaStream_t s_far = nullptr;  // far-field chain (highest priority)
    cudaStream_t s_far2 = nullptr;  // second strength set's far-field chain (log kernel, adjoint; highest priority)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join_far = nullptr, ev_join_far2 = nullptr;
    cudaEvent_t ev_gather = nullptr;  // strengths gathered (fmm_step: P2P waits on it)
    // fmm_step with the evaluation queued behind the list passes: the lists are done (the evaluation waits on
    // it), the build's counters are in h_chk (the host waits on that)
    cudaEvent_t ev_lists = nullptr, ev_chk = nullptr;
    unsigned long long* h_chk = nullptr;  // pinned: status word + counters [0, 5), level bases + needs [8, ...)
    cudaEvent_t ev_t[9] = {};  // phase boundaries of a timed evaluation (fmm_phase_times)
    bool timing_valid = false;

    // persistent evaluation (FMM_FLAG_PERSISTENT): stage table of the device work queue
    void* d_pstage = nullptr;             // device copy of the table
    std::vector<char> h_pstage;           // the table last uploaded
    int npstage = 0;
    long long pstage_total = 0;           // tickets (units) of one evaluation
    unsigned long long* d_pers = nullptr;  // [0] ticket, [1] far-field units done, [2] P2P units done,
                                           // [3] stage + 1 of a queue wait that ran out (0 = none)

    // captured evaluation graph (keyed by the user pointers it bakes in)
    cudaGraphExec_t graph = nullptr;
    std::vector<const void*> p2p_funcs;  // P2P kernels launched by the last evaluation (low graph priority)
    const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};

    // autotuner state (AT3b, Algorithm 4)
    struct Tune {
        double cap = 0.10;      // maximum relative tuning cost
        int window = 3;         // evaluations per decision (minimum taken)
        int period = 8;         // accepted evaluations between moves
        int iter = 0;
        int since_move = 0;
        std::vector<double> win;
        double base_min = 0;    // windowed minimum time of the accepted N_levels
        int accepted = 0;       // accepted N_levels
        int trial = 0;          // N_levels on trial (0 = none)
        int trial_dir = 0;
        int nldir = +1;
        double basetime = 0;    // accumulated time of accepted evaluations
        int accepted_evals = 0;
        double upcost = 0, downcost = 0;
        int wait_up = 0, wait_down = 0;
        int max_levels = 1;
        int rejected = 0;
        double tuning_cost = 0;  // time lost to rejected moves
        // theta moves (Algorithms 2-4): 0.01 x Fibonacci steps, p follows theta through the tolerance
        bool theta_on = false;
        double tol = 1e-6, theta_lo = 0.3, theta_hi = 0.7;
        double theta = 0.5;        // accepted theta
        double theta_trial = 0;    // theta on trial (0 = none)
        int theta_dir = +1;
        int fibcount = 1, fiblength = 3;
        int trial_kind = 0;        // 0 none, 1 N_levels move, 2 theta move
        int next_kind = 1;         // kind of the next move attempt (they alternate)
    } tune;
};

// -------------------------------------------------------------- utilities
void set_error(const std::string& msg);
fmm_status cuda_fail(cudaError_t e, const char* what);

#define FMM_CUDA(call)                                              \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return ::fmm::cuda_fail(_e, #call);  \
    } while (0)

// ------------------------------------------------------------ tree phases
fmm_status build_shape(Tree& t);                                         // host tables + device copies
fmm_status alloc_build(Tree& t);                                         // build scratch / tree arrays
fmm_status alloc_lists(Tree& t);                                         // fixed-capacity lists
fmm_status run_tree_build(Tree& t, const double* d_xy, cudaStream_t s);  // sort, split, geometry
fmm_status run_lists(Tree& t, cudaStream_t s);                           // strong / weak lists, work items
fmm_status run_count(Tree& t, cudaStream_t s, unsigned long long out[2]);
fmm_status alloc_eval(Tree& t, int sets);        // alloc_eval_core + alloc_eval_parts
fmm_status alloc_eval_core(Tree& t, int sets);   // buffers that follow the tree shape and the expansion order
fmm_status alloc_eval_parts(Tree& t);            // partial sums: follow the work-item capacities of the lists
fmm_status run_eval(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s);
fmm_status run_eval_log(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s);  // needs alloc_eval(t, 2)
fmm_status prepare_persistent(Tree& t);  // stage table of the persistent evaluation (not under stream capture)
fmm_status run_eval_persistent(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s);
fmm_status run_backward(Tree& t, const double* d_gamma, const double* d_gphi, double* d_ggamma, double* d_gxy,
                        cudaStream_t s);

// Buffers of one strength set of the evaluation workspace.
struct Bufs {
    void* gam;
    void* near;
    double2* M64;
    float2* M32;
    void* Lm2l;
    double2* L64;
    float2* L32;
    void* p2p_part;
    void* m2l_part;
};
Bufs bufs(Tree& t, int set);
// FP32 path with at least three levels: the deepest level's L2L is folded into L2P (Tree::d_fold_par).
inline bool fold_leaf_l2l(const Tree& t) { return t.path == FMM_PATH_FP32 && t.Lmax >= 3; }
// FP32 path, parent levels whose boxes hold few points: their multipoles by P2M from their own points instead
// of the M2M shift of their children's (the shift of a truncated multipole is exact), which spares the largest
// FP64 shift launches of the upward pass.  Returns 1 (a thread per box: at most 64 points), 2 (a warp per box:
// at most 1024) or 0 (M2M).  A box on level l holds at most max_leaf * 4^(Lmax - 1 - l) points.
inline int p2m_parent_mode(const Tree& t, int l) {
    if (t.path != FMM_PATH_FP32 || t.Lmax < 3 || l < 1) return 0;
    const int up = t.Lmax - 1 - l;  // levels between l and the deepest leaves
    if (up > 8) return 0;
    const long long most = (long long)t.max_leaf << (2 * up);
    return most <= 64 ? 1 : most <= 1024 ? 2 : 0;
}
bool m2l_tc_enabled();
// Weak pairs per M2L work item.  Tensor-core M2L, measured with the row order on the 1e6-point step (ms):
// 64: 3.32, 128: 3.25, 160: 3.23, 192: 3.22, 256: 3.23.  FP64 M2L (one thread per item): 32, 64 and 128 equal.
inline int m2l_item_pairs(const Tree& t) {
    return t.path == FMM_PATH_FP32 && m2l_tc_enabled() ? 192 : 64;
}
fmm_status complete_folded_locals(Tree& t, cudaStream_t s);  // the skipped L2L, for the export of locals
bool refresh_grids(Tree& t);  // true when the P2P / M2L grids changed (the graph must be re-captured)
long long p2p_grid_items(const Tree& t);
long long m2l_grid_items(const Tree& t);
void dispatch_far(Tree& t, const Bufs& B, cudaStream_t s, bool log_kernel = false);
void dispatch_up(Tree& t, const Bufs& B, cudaStream_t s);                          // P2M, M2M (tree only)
void dispatch_down(Tree& t, const Bufs& B, cudaStream_t s, bool log_kernel = false);  // M2L .. L2L (lists)
void launch_gather(Tree& t, const Bufs& B, const double* d_gamma, cudaStream_t s);
void launch_near(Tree& t, const Bufs& B, cudaStream_t s);                      // harmonic P2P + ordered sums
void launch_l2p_near(Tree& t, const Bufs& B, void* d_phi, cudaStream_t s);     // L2P + near + unpermute  // P2M, M2M, M2L, L2L of one strength set

// FP32-path M2L on the tensor cores (m2l_tc.cu); FMM_M2L_TC=0 selects the CUDA-core kernel.
bool m2l_tc_enabled();
fmm_status m2l_tc_prepare(int P);
// Self-tests of the bounded waits (a wait on something that never happens; ST_TIMEOUT expected).
void launch_selftest_mbar(int limit, unsigned* status, cudaStream_t s);
void launch_selftest_lookback(unsigned long long* st, int max_spins, unsigned* status, cudaStream_t s);
void launch_selftest_queue(unsigned long long* ctr, unsigned long long limit_ns, unsigned* status, cudaStream_t s);
void launch_selftest_rcp64(const double* x, int64_t n, double* out, cudaStream_t s);  // once per compiled order, before launches (and graph capture)
void launch_m2l_tc(const Tree& t, const float2* M32, float2* Lm2l, float2* part, bool log_kernel, cudaStream_t s);

// Autotuner (host).
int default_nlevels(int64_t n, int p, int path);

int tune_step(Tree::Tune& u, double time_s);
int p_for_tolerance(double tol, double theta);
double tune_theta(const Tree::Tune& u);  // theta to use next (accepted or on trial)

// Smallest compiled expansion order >= p (kernels are templates on the order).
int compiled_order(int p);

}  // namespace fmm

// The opaque handle of the C ABI.
struct fmm_tree {
    fmm::Tree t;
};

// ---------------------------------------------------------------- device
#ifdef __CUDACC__
namespace fmm {

// C(n,k) by the multiplicative formula; exact in double for n <= 62.
__host__ __device__ constexpr double binom_d(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    if (k > n - k) k = n - k;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * double(n - k + i) / double(i);
    return r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a*b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x in FP64 for a positive x: the hardware's approximate reciprocal
// (rcp.approx.ftz.f64) refined by two Newton-Raphson steps y <- y + y (1 - x y)
// (Newton's method on f(y) = 1/y - x: each step squares the relative error),
// within about one ulp of the correctly rounded value at 5 instructions.  x
// below the smallest normal double (a pair closer than ~1e-154) gives 0: such
// pairs are treated as coincident.
__device__ __forceinline__ double rcp_nr64(double x) {
    if (!(x >= 2.2250738585072014e-308)) return 0.0;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Packed 2 x FP32 (f32x2) arithmetic: the low 32 bits hold the first value.
// Work item of P2P ticket t in the row order (see Tree::d_p2p_rows): nheavy = rows taken from the front.
__device__ __forceinline__ int p2p_row_item(int t, const int32_t* __restrict__ rows, unsigned long long nheavy,
                                            long long cap) {
    return (unsigned long long)t < nheavy ? rows[t] : rows[cap - 1 - ((long long)t - (long long)nheavy)];
}

typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2pk(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2upk(f2x v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x f2add(f2x a, f2x b) {
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2sub(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2mul(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2fma(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Index of the segment containing position i: largest k with start[k] <= i.
__device__ __forceinline__ int find_seg(const int32_t* __restrict__ start, int K, int i) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace fmm
#endif
