// Tree build of the balanced adaptive FMM on the device (Sec. 2.2-2.3 of the
// paper: a pyramid of full levels, every box split into four at exact medians,
// x first and then y within each half) and the strong / weak coupling lists of
// Sec. 2.1 with the theta-criterion of eq (2.3).
//
// Design: both coordinates are sorted once by an LSD radix sort on
// order-preserving 64-bit keys with the input index as tie-break (stable).
// After that a median split never compares coordinates again: every box keeps
// its points as two lists, one in (x, index) order and one in (y, index) order.
// The x-split of a box is a contiguous cut of its x-list; the y-list is then
// stably partitioned by the side flags of that cut (segmented scan + scatter).
// The y-split of each half is the mirror image.  Bounding boxes come for free
// from the first/last entries of the two lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "fmm_internal.cuh"

namespace fmm {

// ================================================================ shape (host)

static int64_t lvl_off(int l) {  // boxes on levels < l of one instance
    int64_t s = 0, w = 1;
    for (int i = 0; i < l; ++i) { s += w; w *= 4; }
    return s;
}

template <typename T>
static fmm_status upload(T** dst, const std::vector<T>& v) {
    if (*dst) { cudaFree(*dst); *dst = nullptr; }
    size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    FMM_CUDA(cudaMalloc((void**)dst, bytes));
    if (!v.empty()) FMM_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FMM_OK;
}

static void free_list(LevelList& l) {
    if (l.d_ids) cudaFree(l.d_ids);
    l.d_ids = nullptr;
    l.count = 0;
}
static void free_seg(SegTable& s) {
    if (s.d_start) cudaFree(s.d_start);
    if (s.d_nzero) cudaFree(s.d_nzero);
    if (s.d_obefore) cudaFree(s.d_obefore);
    s = SegTable();
}

// Flag-1 positions before each segment: segment j holds (length - nzero) of them.
static std::vector<int32_t> ones_before(const std::vector<int32_t>& start, const std::vector<int32_t>& nzero) {
    std::vector<int32_t> ob(nzero.size());
    int64_t acc = 0;
    for (size_t k = 0; k < nzero.size(); ++k) {
        ob[k] = (int32_t)acc;
        acc += (start[k + 1] - start[k]) - nzero[k];
    }
    return ob;
}

// Point ranges, parents and children of every box follow from the instance
// sizes alone: a box of n points gives its x-halves floor(n/2) and ceil(n/2)
// points, and each half gives its y-halves the floor / ceil of its own count.
fmm_status build_shape(Tree& t) {
    const int B = t.ninst;
    t.Lmax = 1;
    t.inst_box_off.assign(B + 1, 0);
    for (int b = 0; b < B; ++b) {
        t.Lmax = std::max(t.Lmax, t.inst_levels[b]);
        t.inst_box_off[b + 1] = t.inst_box_off[b] + lvl_off(t.inst_levels[b]);
    }
    t.nbox = t.inst_box_off[B];
    if (t.nbox >= (int64_t(1) << 30)) { set_error("too many boxes"); return FMM_ERR_INVALID_ARG; }
    t.h_bstart.assign(t.nbox, 0);
    t.h_bcount.assign(t.nbox, 0);
    t.h_parent.assign(t.nbox, -1);
    t.h_child0.assign(t.nbox, -1);
    t.h_inst.assign(t.nbox, 0);
    t.h_level_boxes.assign(t.Lmax, {});
    std::vector<std::vector<int32_t>> lvl_par(t.Lmax);
    t.h_leaves.clear();
    for (int b = 0; b < B; ++b) {
        const int L = t.inst_levels[b];
        const int64_t bo = t.inst_box_off[b];
        t.h_bstart[bo] = (int32_t)t.inst_pt_off[b];
        t.h_bcount[bo] = (int32_t)(t.inst_pt_off[b + 1] - t.inst_pt_off[b]);
        for (int l = 0; l < L; ++l) {
            const int64_t nb = int64_t(1) << (2 * l);
            for (int64_t i = 0; i < nb; ++i) {
                const int64_t g = bo + lvl_off(l) + i;
                t.h_inst[g] = b;
                t.h_level_boxes[l].push_back((int32_t)g);
                if (l + 1 == L) { t.h_leaves.push_back((int32_t)g); continue; }
                lvl_par[l].push_back((int32_t)g);
                const int32_t s = t.h_bstart[g], n = t.h_bcount[g];
                const int32_t nl = n / 2, nr = n - nl;
                const int64_t c0 = bo + lvl_off(l + 1) + 4 * i;
                t.h_child0[g] = (int32_t)c0;
                const int32_t cs[4] = {s, s + nl / 2, s + nl, s + nl + nr / 2};
                const int32_t cn[4] = {nl / 2, nl - nl / 2, nr / 2, nr - nr / 2};
                for (int c = 0; c < 4; ++c) {
                    t.h_bstart[c0 + c] = cs[c];
                    t.h_bcount[c0 + c] = cn[c];
                    t.h_parent[c0 + c] = (int32_t)g;
                }
            }
        }
    }
    t.nleaf = (int64_t)t.h_leaves.size();
    t.max_leaf = 1;
    for (int32_t lf : t.h_leaves) t.max_leaf = std::max(t.max_leaf, (int)t.h_bcount[lf]);
    t.leaf_cap = leaf_capacity(t.max_leaf);
    if ((t.nleaf + 1) * (int64_t)t.leaf_cap >= (int64_t(1) << 31)) {
        set_error("too many P2P slots (leaves x leaf capacity)");
        return FMM_ERR_INVALID_ARG;
    }
    std::vector<int32_t> pslot(t.nbox, -1);
    for (int64_t q = 0; q < t.nleaf; ++q) pslot[t.h_leaves[q]] = (int32_t)(q * t.leaf_cap);
    fmm_status st;
    if ((st = upload(&t.d_pslot, pslot))) return st;
    if ((st = upload(&t.d_bstart, t.h_bstart))) return st;
    if ((st = upload(&t.d_bcount, t.h_bcount))) return st;
    if ((st = upload(&t.d_parent, t.h_parent))) return st;
    if ((st = upload(&t.d_child0, t.h_child0))) return st;
    {
        std::vector<int32_t> fp(t.nbox, -1);
        if (t.Lmax >= 3)
            for (int32_t g : t.h_level_boxes[t.Lmax - 1]) fp[g] = t.h_parent[g];
        if ((st = upload(&t.d_fold_par, fp))) return st;
    }
    if ((st = upload(&t.d_inst, t.h_inst))) return st;
    if ((st = upload(&t.d_inst_ptoff, t.inst_pt_off))) return st;
    if ((st = upload(&t.d_inst_boxoff, t.inst_box_off))) return st;
    for (auto& l : t.level_boxes) free_list(l);
    for (auto& l : t.level_parents) free_list(l);
    free_list(t.leaves);
    t.level_boxes.assign(t.Lmax, {});
    t.level_parents.assign(t.Lmax, {});
    for (int l = 0; l < t.Lmax; ++l) {
        t.level_boxes[l].count = (int)t.h_level_boxes[l].size();
        if ((st = upload(&t.level_boxes[l].d_ids, t.h_level_boxes[l]))) return st;
        t.level_parents[l].count = (int)lvl_par[l].size();
        if ((st = upload(&t.level_parents[l].d_ids, lvl_par[l]))) return st;
    }
    t.leaves.count = (int)t.nleaf;
    if ((st = upload(&t.leaves.d_ids, t.h_leaves))) return st;
    {
        std::vector<int32_t> ls(t.nleaf + 1);
        for (int64_t i = 0; i < t.nleaf; ++i) ls[i] = t.h_bstart[t.h_leaves[i]];
        ls[t.nleaf] = (int32_t)t.n;
        if ((st = upload(&t.d_leaf_start, ls))) return st;
    }

    // partition segment tables, one x-stage and one y-stage per level
    for (auto& s : t.seg_x) free_seg(s);
    for (auto& s : t.seg_y) free_seg(s);
    t.seg_x.assign(std::max(t.Lmax - 1, 0), {});
    t.seg_y.assign(std::max(t.Lmax - 1, 0), {});
    int64_t maxK = 1;
    for (int l = 0; l + 1 < t.Lmax; ++l) {
        std::vector<int32_t> xs, xz, ys, yz;
        for (int b = 0; b < B; ++b) {
            const int L = t.inst_levels[b];
            const int32_t ps = (int32_t)t.inst_pt_off[b], pn = (int32_t)(t.inst_pt_off[b + 1] - t.inst_pt_off[b]);
            if (l + 1 >= L) {  // this instance is already at its leaves: one inert segment
                xs.push_back(ps); xz.push_back(pn);
                ys.push_back(ps); yz.push_back(pn);
                continue;
            }
            const int64_t bo = t.inst_box_off[b] + lvl_off(l);
            for (int64_t i = 0; i < (int64_t(1) << (2 * l)); ++i) {
                const int32_t s = t.h_bstart[bo + i], n = t.h_bcount[bo + i];
                const int32_t nl = n / 2, nr = n - nl;
                xs.push_back(s); xz.push_back(nl);
                ys.push_back(s); yz.push_back(nl / 2);
                ys.push_back(s + nl); yz.push_back(nr / 2);
            }
        }
        xs.push_back((int32_t)t.n);
        ys.push_back((int32_t)t.n);
        t.seg_x[l].K = (int)xz.size();
        t.seg_y[l].K = (int)yz.size();
        maxK = std::max<int64_t>(maxK, (int64_t)std::max(xz.size(), yz.size()));
        if ((st = upload(&t.seg_x[l].d_start, xs))) return st;
        if ((st = upload(&t.seg_x[l].d_nzero, xz))) return st;
        if ((st = upload(&t.seg_y[l].d_start, ys))) return st;
        if ((st = upload(&t.seg_y[l].d_nzero, yz))) return st;
        if ((st = upload(&t.seg_x[l].d_obefore, ones_before(xs, xz)))) return st;
        if ((st = upload(&t.seg_y[l].d_obefore, ones_before(ys, yz)))) return st;
    }
    t.segs_cap = maxK;
    // first level whose splitting boxes all fit one CTA of the subtree kernel
    t.l0 = t.Lmax - 1;
    for (int l = 0; l + 1 < t.Lmax; ++l) {
        int mx = 0;
        for (int32_t g : lvl_par[l]) mx = std::max(mx, (int)t.h_bcount[g]);
        if (mx <= kSubMax) {
            t.l0 = l;
            break;
        }
    }
    if ((st = upload(&t.d_inst_levels, t.inst_levels))) return st;
    return FMM_OK;
}

// ============================================================== radix sort

// Order-preserving key of a double (+0 and -0 map to the same key).
__device__ __forceinline__ uint64_t order_key(double v) {
    if (v == 0.0) v = 0.0;
    uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_keys(const double2* __restrict__ xy, int n, uint64_t* kx, uint64_t* ky, int32_t* vx, int32_t* vy,
                       unsigned* status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 p = xy[i];
    if (!isfinite(p.x) || !isfinite(p.y)) atomicOr(status, ST_NONFINITE);
    kx[i] = order_key(p.x);
    ky[i] = order_key(p.y);
    vx[i] = i;
    vy[i] = i;
}

// Instance index of each sorted entry (batched trees): the digit source of the
// two final stable passes that group the points by instance.
__global__ void k_inst_keys(const int32_t* __restrict__ vx, const int32_t* __restrict__ vy,
                            const int64_t* __restrict__ ptoff, int ninst, int n, uint64_t* kx, uint64_t* ky) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int s = 0; s < 2; ++s) {
        int v = s ? vy[i] : vx[i];
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (ptoff[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        (s ? ky : kx)[i] = (uint64_t)lo;
    }
}

// As block_excl_scan without the closing barrier: the caller passes a barrier before wsum is written again.
__device__ __forceinline__ int block_excl_scan_nb(int v, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int ws = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        wsum[lane] = ws;
    }
    __syncthreads();
    total = wsum[nw - 1];
    return x - v + (w ? wsum[w - 1] : 0);
}

__device__ __forceinline__ int block_excl_scan(int v, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int ws = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        wsum[lane] = ws;
    }
    __syncthreads();
    total = wsum[nw - 1];
    int r = x - v + (w ? wsum[w - 1] : 0);
    __syncthreads();
    return r;
}

// Per-tile digit histograms of both sorts (blockIdx.y = which sort).
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint64_t* __restrict__ k0,
                                                            const uint64_t* __restrict__ k1, int n, int shift, int T,
                                                            int32_t* hist /*[2][256][T]*/, int32_t* tot /*[2][256]*/) {
    __shared__ int h[256];
    const int s = blockIdx.y, t = blockIdx.x;
    const uint64_t* k = s ? k1 : k0;
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int r = 0; r < kSortRounds; ++r) {
        int i = t * kSortTile + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(int)((k[i] >> shift) & 255u)], 1);
    }
    __syncthreads();
    int c = h[threadIdx.x];
    hist[((size_t)s * 256 + threadIdx.x) * T + t] = c;
    if (c) atomicAdd(&tot[s * 256 + threadIdx.x], c);
}

// Exclusive offsets: block (d, s) scans digit d's tile counts and adds the
// number of keys with a smaller digit.
__global__ void __launch_bounds__(1024) k_sort_scan(const int32_t* __restrict__ hist, const int32_t* __restrict__ tot,
                                                    int T, int32_t* off) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int d = blockIdx.x, s = blockIdx.y;
    if (threadIdx.x < 32) {
        int acc = 0;
        for (int e = threadIdx.x; e < d; e += 32) acc += tot[s * 256 + e];
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) base = acc;
    }
    __syncthreads();
    const int32_t* hrow = hist + ((size_t)s * 256 + d) * T;
    int32_t* orow = off + ((size_t)s * 256 + d) * T;
    int carry = base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c0 = 0; c0 < T; c0 += 1024) {
        int i = c0 + threadIdx.x;
        int v = i < T ? hrow[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int ws = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            wsum[lane] = ws;
        }
        __syncthreads();
        int excl = x - v + (w ? wsum[w - 1] : 0);
        if (i < T) orow[i] = carry + excl;
        int total = wsum[31];
        __syncthreads();
        carry += total;
    }
}

// Global digit counts of all 8 LSD passes of both sorts in one read of the
// keys (a digit's count does not depend on the order): ghist[s][pass][digit].
// P0 = first pass counted (4: the high halves only).  FROM_XY: the keys are
// formed here from the points (and non-finite coordinates reported) instead of
// read.
template <int P0, bool FROM_XY>
__global__ void __launch_bounds__(kSortThreads) k_sort_ghist(const uint64_t* __restrict__ k0,
                                                             const uint64_t* __restrict__ k1, int n,
                                                             unsigned* __restrict__ ghist,
                                                             const double2* __restrict__ xy, unsigned* status) {
    pdl_wait();
    __shared__ unsigned h[8][256];
    const int s = blockIdx.y;
    const uint64_t* k = s ? k1 : k0;
    for (int e = threadIdx.x; e < 8 * 256; e += kSortThreads) (&h[0][0])[e] = 0;
    __syncthreads();
    for (int r = 0; r < kSortRounds; ++r) {
        const int i = blockIdx.x * kSortTile + r * kSortThreads + threadIdx.x;
        if (i < n) {
            uint64_t key;
            if constexpr (FROM_XY) {
                const double c = s ? xy[i].y : xy[i].x;
                if (!isfinite(c)) atomicOr(status, ST_NONFINITE);
                key = order_key(c);
            } else {
                key = k[i];
            }
#pragma unroll
            for (int p = P0; p < 8; ++p) atomicAdd(&h[p][(int)((key >> (8 * p)) & 255u)], 1u);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 8 * 256; e += kSortThreads) {
        const unsigned c = (&h[0][0])[e];
        if (c) atomicAdd(ghist + (size_t)s * 8 * 256 + e, c);
    }
}

// Stable scatter of one 8-bit digit.  Warp w of a tile owns its 256
// consecutive keys (lane l holds keys w*256 + 32 r + l, r = 0..7, loaded up
// front); each warp ranks its keys round by round with match_any and a
// warp-private digit counter, so the rounds need only warp synchronisation.
// One exclusive pass over the warps per digit then gives every key its rank
// among the tile's keys of its digit (input order: stable).  The tile is
// reordered by digit in shared memory and written back so that consecutive
// threads store consecutive keys of a digit: each digit's run of the tile is
// one contiguous piece of the output.
// Where a tile's run of digit d starts in the output:
//   ONESWEEP false: off[s][d][t], from the per-tile histograms and their scan;
//   ONESWEEP true:  the digit's global base (from the pass's global counts)
//     plus the count of digit d in the tiles before t, by a decoupled
//     look-back (thread d publishes the tile's count of digit d, then walks
//     back over earlier tiles' words until one holds an inclusive prefix).
//     Tiles are taken in ticket order, so a tile only waits on tiles that
//     running CTAs hold; every wait is bounded (ST_TIMEOUT).  Status words
//     stat[s][t][d]: bits 30-31 = 0 (not yet), 1 (tile count), 2 (inclusive
//     prefix); bits 0-29 = the count.
constexpr unsigned kSAgg = 1u << 30, kSIncl = 2u << 30, kSVal = (1u << 30) - 1;
constexpr int kSortSpins = 1 << 21;  // bound on the look-back's waits for one tile
// earlier tiles one look-back round reads; measured on the 1e6-point build: 4 beats 1, 8 and 16
constexpr int kSortLook = 4;
template <bool ONESWEEP, bool FROM_XY = false>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t* __restrict__ ki0,
                                                               const int32_t* __restrict__ vi0,
                                                               const uint64_t* __restrict__ ki1,
                                                               const int32_t* __restrict__ vi1, uint64_t* ko0,
                                                               int32_t* vo0, uint64_t* ko1, int32_t* vo1, int n,
                                                               int shift, int T, const int32_t* __restrict__ off,
                                                               const unsigned* __restrict__ ghist, unsigned* stat,
                                                               unsigned* ticket, unsigned* status,
                                                               const double2* __restrict__ xy = nullptr) {
    pdl_wait();
    constexpr int W = kSortThreads / 32;
    __shared__ int whist[W][257];  // per-warp digit counts, then their exclusive prefix over warps
    __shared__ int base[256];      // global position of the tile's first key of each digit
    __shared__ int tstart[257];    // first tile-local slot of each digit
    __shared__ int wsum[32];
    __shared__ uint64_t skey[kSortTile];
    __shared__ int sval[kSortTile];
    __shared__ int sh_t;
    const int s = blockIdx.y, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    int t = blockIdx.x;
    if constexpr (ONESWEEP) {
        if (tid == 0) sh_t = (int)atomicAdd(ticket + s, 1u);
        __syncthreads();
        t = sh_t;
        if (t >= T) return;  // CTA-uniform (the grid has exactly T CTAs per sort)
    } else {
        base[tid] = off[((size_t)s * 256 + tid) * T + t];
    }
    const uint64_t* ki = s ? ki1 : ki0;
    const int32_t* vi = s ? vi1 : vi0;
    uint64_t* ko = s ? ko1 : ko0;
    int32_t* vo = s ? vo1 : vo0;
#pragma unroll
    for (int j = 0; j < 257; j += 32)
        if (j + lane < 257) whist[warp][j + lane] = 0;
    uint64_t key[kSortRounds];
    int val[kSortRounds], rank[kSortRounds], dig[kSortRounds];
    const int i0 = t * kSortTile + warp * (32 * kSortRounds) + lane;
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int i = i0 + 32 * r;
        const bool valid = i < n;
        if constexpr (FROM_XY) {  // the first pass: keys from the points, values = input indices
            key[r] = valid ? order_key(s ? xy[i].y : xy[i].x) : 0;
            val[r] = i;
        } else {
            key[r] = valid ? ki[i] : 0;
            val[r] = valid ? vi[i] : 0;
        }
        dig[r] = valid ? (int)((key[r] >> shift) & 255u) : 256;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int d = dig[r];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = whist[warp][d];
        rank[r] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (lane == __ffs(peers) - 1) whist[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    int cnt = 0;
    {  // thread = digit: exclusive prefix of the digit's count over the warps
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int c = whist[w][tid];
            whist[w][tid] = cnt;
            cnt += c;
        }
    }
    if constexpr (ONESWEEP) {
        // the digit's global base: exclusive prefix of the pass's global counts over the digits
        const unsigned* gh = ghist + (size_t)s * 8 * 256;
        int gtot;
        const int gb = block_excl_scan((int)gh[tid], wsum, gtot);
        unsigned* st = stat + (size_t)s * T * 256;
        volatile unsigned* me = st + (size_t)t * 256 + tid;
        unsigned excl = 0;
        if (t == 0) {
            *me = kSIncl | (unsigned)cnt;
        } else {
            *me = kSAgg | (unsigned)cnt;
            // kSortLook earlier tiles per round (independent loads): the nearest inclusive prefix among them
            // ends the walk, every tile up to it must have published
            int j = t - 1, spins = 0;
            while (true) {
                unsigned v[kSortLook];
#pragma unroll
                for (int u = 0; u < kSortLook; ++u) {
                    const int q = j - u;
                    v[u] = q >= 0 ? (unsigned)*((volatile unsigned*)(st + (size_t)q * 256 + tid))
                                  : (unsigned)kSIncl;  // before tile 0: an empty prefix
                }
                int first = kSortLook;
#pragma unroll
                for (int u = kSortLook - 1; u >= 0; --u)
                    if ((v[u] & ~kSVal) == kSIncl) first = u;
                bool notready = false;
                unsigned sum = 0;
#pragma unroll
                for (int u = 0; u < kSortLook; ++u) {
                    if (u <= first) {
                        notready |= (v[u] & ~kSVal) == 0;
                        sum += v[u] & kSVal;
                    }
                }
                if (notready) {
                    if (++spins > kSortSpins) {
                        atomicOr(status, ST_TIMEOUT);
                        break;
                    }
                    continue;
                }
                excl += sum;
                if (first < kSortLook) break;
                j -= kSortLook;
            }
            *me = kSIncl | (excl + (unsigned)cnt);
        }
        base[tid] = gb + (int)excl;
    }
    int total;
    const int st0 = block_excl_scan(cnt, wsum, total);  // first local slot of digit tid (contains barriers)
    tstart[tid] = st0;
    if (tid == 0) tstart[256] = total;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int d = dig[r];
        if (d < 256) {
            const int slot = tstart[d] + whist[warp][d] + rank[r];
            skey[slot] = key[r];
            sval[slot] = val[r];
        }
    }
    __syncthreads();
    for (int j = tid; j < total; j += kSortThreads) {
        const uint64_t k = skey[j];
        const int d = (int)((k >> shift) & 255u);
        const int pos = base[d] + (j - tstart[d]);
        if (pos >= 0 && pos < n) {
            ko[pos] = k;
            vo[pos] = sval[j];
        } else {
            atomicOr(status, ST_INTERNAL);
        }
    }
}

static inline int nblk(int64_t n, int b) { return (int)std::max<int64_t>((n + b - 1) / b, 1); }

// One LSD pass over both sorts: (keys,vals)[src..src+1] -> [dst..dst+1].
static fmm_status sort_pass(Tree& t, cudaStream_t s, int src, int dst, int shift) {
    const int n = (int)t.n;
    const int T = nblk(n, kSortTile);
    FMM_CUDA(cudaMemsetAsync(t.d_sort_tot, 0, 2 * 256 * sizeof(int32_t), s));
    dim3 g(T, 2);
    k_sort_hist<<<g, kSortThreads, 0, s>>>(t.d_keys[src], t.d_keys[src + 1], n, shift, T, t.d_sort_hist,
                                           t.d_sort_tot);
    k_sort_scan<<<dim3(256, 2), 1024, 0, s>>>(t.d_sort_hist, t.d_sort_tot, T, t.d_sort_off);
    k_sort_scatter<false><<<g, kSortThreads, 0, s>>>(t.d_keys[src], t.d_vals[src], t.d_keys[src + 1],
                                                     t.d_vals[src + 1], t.d_keys[dst], t.d_vals[dst],
                                                     t.d_keys[dst + 1], t.d_vals[dst + 1], n, shift, T, t.d_sort_off,
                                                     nullptr, nullptr, nullptr, t.d_status);
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

// Runs of equal high key halves after the high-half passes.  The passes are
// stable, so inside a run the entries are in input order; the full order is by
// (key, input index), i.e. by (key, position in the run).  Each entry counts
// the entries of its run that precede it in that order and writes its value
// (input index) to run start + count in the output; an entry outside any run
// keeps its place.  Runs longer than kSortRunMax are reported (ST_SORT_RUN) and
// copied unchanged (a permutation all the same: later kernels index with it),
// and the host rebuilds with all 64 bits.  blockIdx.y = which sort; only the
// values are written (the tree build needs the order, not the keys).
constexpr int kSortRunMax = 16;
__global__ void __launch_bounds__(256) k_sort_runs(const uint64_t* __restrict__ k0, const int32_t* __restrict__ v0,
                                                   const uint64_t* __restrict__ k1, const int32_t* __restrict__ v1,
                                                   int32_t* __restrict__ o0, int32_t* __restrict__ o1, int n,
                                                   uint8_t* __restrict__ side0, const int32_t* __restrict__ nz0,
                                                   unsigned* status) {
    pdl_wait();
    const uint64_t* key = blockIdx.y ? k1 : k0;
    const int32_t* val = blockIdx.y ? v1 : v0;
    int32_t* out = blockIdx.y ? o1 : o0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the entry and both neighbours at once: most entries are not in a run
    const uint64_t ki = key[i];
    const uint64_t kp = i > 0 ? key[i - 1] : 0, kn = i + 1 < n ? key[i + 1] : 0;
    const int32_t vi = val[i];
    const unsigned hi = (unsigned)(ki >> 32);
    const bool prev = i > 0 && (unsigned)(kp >> 32) == hi, next = i + 1 < n && (unsigned)(kn >> 32) == hi;
    const bool mark = side0 != nullptr && blockIdx.y == 0;  // x sort: also the side flags of the root's x cut
    if (!prev && !next) {
        out[i] = vi;
        if (mark) side0[vi] = (uint8_t)(i >= *nz0);
        return;
    }
    int s = prev ? i - 1 : i;
    while (s > 0 && i - s < kSortRunMax && (unsigned)(key[s - 1] >> 32) == hi) --s;
    int e = next ? i + 2 : i + 1;
    while (e < n && e - s <= kSortRunMax && (unsigned)(key[e] >> 32) == hi) ++e;
    if (e - s > kSortRunMax || (s > 0 && (unsigned)(key[s - 1] >> 32) == hi)) {
        if ((i & 15) == 0) atomicOr(status, ST_SORT_RUN);  // a long run holds such an i
        out[i] = vi;
        if (mark) side0[vi] = (uint8_t)(i >= *nz0);
        return;
    }
    int rank = 0;
    for (int j = s; j < e; ++j) {
        const uint64_t kj = key[j];
        rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
    }
    out[s + rank] = vi;
    if (mark) side0[vi] = (uint8_t)(s + rank >= *nz0);
}

// Words of the onesweep scratch for n points.
static size_t sort_scratch_words(int64_t n) {
    const int64_t T = (n + kSortTile - 1) / kSortTile;
    return (size_t)(2 * 8 * 256 + 16 + 8 * 2 * T * 256);
}

// LSD passes over the 64-bit coordinate keys of both sorts: one kernel for the
// global digit counts of every pass, then one onesweep kernel per pass.  full:
// all 8 passes; otherwise the 4 passes of the high halves and then k_sort_runs
// for the runs of equal high halves (short for point sets without heavy
// repetition of the leading 20 mantissa bits; a longer run is reported and the
// host rebuilds with full = true).  Both give the order by (key, input index).
// Scratch: d_sort_os = global counts [2][8][256], tickets [8][2], tile status
// words [8][2][T][256]; zeroed once per build.  *res: the buffer pair that
// holds the sorted values (0: 0/1, 2: 2/3).
static fmm_status sort_coordinates(Tree& t, cudaStream_t s, const double2* xy, bool full, int* res, uint8_t* side0,
                                   const int32_t* nz0) {
    const int n = (int)t.n;
    const int T = nblk(n, kSortTile);
    unsigned* gh = t.d_sort_os;
    unsigned* tk = gh + 2 * 8 * 256;
    unsigned* stat = tk + 16;
    FMM_CUDA(cudaMemsetAsync(gh, 0, sort_scratch_words(n) * sizeof(unsigned), s));
    dim3 g(T, 2);
    if (full)
        launch_dep(false, k_sort_ghist<0, true>, g, kSortThreads, 0, s, nullptr, nullptr, n, gh, xy, t.d_status);
    else
        launch_dep(false, k_sort_ghist<4, true>, g, kSortThreads, 0, s, nullptr, nullptr, n, gh, xy, t.d_status);
    int src = 0;
    const int p0 = full ? 0 : 4;
    for (int pass = p0; pass < 8; ++pass) {  // an even number of passes: the result is in buffers 0/1
        const int dst = 2 - src;
        if (pass == p0)  // the first pass forms the keys from the points
            launch_dep(true, k_sort_scatter<true, true>, g, kSortThreads, 0, s,
                       nullptr, nullptr, nullptr, nullptr, t.d_keys[dst], t.d_vals[dst], t.d_keys[dst + 1],
                       t.d_vals[dst + 1], n, 8 * pass, T, nullptr, gh + pass * 256, stat + (size_t)pass * 2 * T * 256,
                       tk + 2 * pass, t.d_status, xy);
        else
            launch_dep(true, k_sort_scatter<true>, g, kSortThreads, 0, s,
                       t.d_keys[src], t.d_vals[src], t.d_keys[src + 1], t.d_vals[src + 1], t.d_keys[dst],
                       t.d_vals[dst], t.d_keys[dst + 1], t.d_vals[dst + 1], n, 8 * pass, T, nullptr, gh + pass * 256,
                       stat + (size_t)pass * 2 * T * 256, tk + 2 * pass, t.d_status, nullptr);
        FMM_CUDA(cudaGetLastError());
        src = dst;
    }
    *res = 0;
    if (!full) {  // the runs: values 0/1 -> 2/3
        launch_dep(true, k_sort_runs, dim3(nblk(n, 256), 2), 256, 0, s,
                   t.d_keys[0], t.d_vals[0], t.d_keys[1], t.d_vals[1], t.d_vals[2], t.d_vals[3], n, side0, nz0,
                   t.d_status);
        FMM_CUDA(cudaGetLastError());
        *res = 2;
    }
    return FMM_OK;
}

// ================================================================ geometry

// Box geometry from the first/last entries of the box's x- and y-lists:
// centre = midpoint of the tight bounding box, radius = half its diagonal
// (FP64 with explicit rounding, no contraction, so values are reproducible).
// One level's boxes (ids[0..cnt)) with that level's lists X and Y.
struct GeomArgs {
    const int32_t* ids;
    int cnt;
    const int32_t* X;
    const int32_t* Y;
    const double2* xy;
    const int32_t* bstart;
    const int32_t* bcount;
    const int32_t* inst;
    const int64_t* inst_box_off;
    double2* center;
    double* radius;
    double* rho;
    float4* chl;
    float* rho32;
    float* rad32;
    int is_root_level;
};

__device__ __forceinline__ void geom_box(const GeomArgs& g, int q) {
    const int b = g.ids[q];
    const int s = g.bstart[b], e = s + g.bcount[b] - 1;
    const double x0 = g.xy[g.X[s]].x, x1 = g.xy[g.X[e]].x;
    const double y0 = g.xy[g.Y[s]].y, y1 = g.xy[g.Y[e]].y;
    const double cx = __dmul_rn(0.5, __dadd_rn(x0, x1));
    const double cy = __dmul_rn(0.5, __dadd_rn(y0, y1));
    const double dx = __dsub_rn(x1, x0), dy = __dsub_rn(y1, y0);
    const double r = __dmul_rn(0.5, __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))));
    g.center[b] = make_double2(cx, cy);
    g.radius[b] = r;
    g.rad32[b] = __double2float_rn(r);
    // Scale radius of the expansions: the bbox radius, floored at 2^-24 of the
    // instance's root radius so that a box of coincident points still keeps a
    // usable local-expansion derivative; rounded to FP32 so both precisions
    // scale by the same number.
    double ox = cx, oy = cy, rfloor = 0.0;
    if (!g.is_root_level) {
        const int root = (int)g.inst_box_off[g.inst[b]];
        const double2 o = g.center[root];
        ox = o.x;
        oy = o.y;
        rfloor = ldexp(g.radius[root], -24);
    }
    const double rs = r > rfloor ? r : rfloor;
    const float r32 = rs >= 1e-30 ? __double2float_rn(rs) : 0.0f;
    g.rho32[b] = r32;
    g.rho[b] = (double)r32;
    const double ex = __dsub_rn(cx, ox), ey = __dsub_rn(cy, oy);
    const float hx = __double2float_rn(ex), hy = __double2float_rn(ey);
    g.chl[b] = make_float4(hx, hy, __double2float_rn(__dsub_rn(ex, (double)hx)),
                           __double2float_rn(__dsub_rn(ey, (double)hy)));
}

// ======================================================= segmented partition

// Side flags of a contiguous cut: entry at position i of list A goes to side 1
// when its offset inside its segment is >= nzero of that segment.
__global__ void k_mark(const int32_t* __restrict__ A, int n, const int32_t* __restrict__ start,
                       const int32_t* __restrict__ nzero, int K, uint8_t* side) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = find_seg(start, K, i);
    side[A[i]] = (uint8_t)((i - start[k]) >= nzero[k]);
}


constexpr unsigned long long kLAgg = 1ull << 62, kLIncl = 2ull << 62, kLVal = (1ull << 62) - 1;
constexpr int kLookbackSpins = 1 << 21;

__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Decoupled look-back by one full warp: publishes tile t's aggregate, then
// sums the counts of the preceding tiles 32 at a time (lane i reads tile
// j - i) down to the nearest inclusive prefix, and publishes t's inclusive
// prefix.  Returns the exclusive prefix of tile t (all lanes).  Bounded: after
// kLookbackSpins rounds that met a tile with nothing published it sets
// ST_TIMEOUT and returns what it has.
__device__ unsigned long long warp_lookback(unsigned long long* st, long long t, unsigned long long agg,
                                            unsigned* status, int max_spins = kLookbackSpins) {
    const int lane = threadIdx.x & 31;
    if (t == 0) {
        if (lane == 0) st_volatile(st, kLIncl | agg);
        return 0;
    }
    if (lane == 0) st_volatile(st + t, kLAgg | agg);
    unsigned long long excl = 0;
    long long j = t - 1;
    int spins = 0;
    while (true) {
        const long long q = j - lane;
        const unsigned long long v = q >= 0 ? ld_volatile(st + q) : kLIncl;  // before tile 0: an empty prefix
        const unsigned long long fl = v & ~kLVal;
        const unsigned incl = __ballot_sync(0xffffffffu, fl == kLIncl);
        const unsigned notready = __ballot_sync(0xffffffffu, fl == 0);
        const int first = incl ? __ffs(incl) - 1 : 32;  // nearest inclusive prefix in this window
        const unsigned need = first == 32 ? 0xffffffffu : (first == 31 ? 0xffffffffu : ((2u << first) - 1u));
        if (notready & need) {
            if (++spins > max_spins) {
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                break;
            }
            continue;
        }
        unsigned long long x = lane <= first ? (v & kLVal) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        excl += x;
        if (first < 32) break;
        j -= 32;
    }
    if (lane == 0) st_volatile(st + t, kLIncl | (excl + agg));
    return excl;
}

// Self-test of the bounded look-back: tile 1 waits on tile 0, which never
// publishes (its status word stays zero); the wait must give up after
// `max_spins` rounds and report ST_TIMEOUT.
__global__ void k_selftest_lookback(unsigned long long* st, int max_spins, unsigned* status) {
    warp_lookback(st, 1, 5ull, status, max_spins);
}
void launch_selftest_lookback(unsigned long long* st, int max_spins, unsigned* status, cudaStream_t s) {
    k_selftest_lookback<<<1, 32, 0, s>>>(st, max_spins, status);
}

// Segment search over starts in shared or global memory (generic pointer).
__device__ __forceinline__ int find_seg_any(const int32_t* start, int K, int i) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
constexpr int kPartSegSmem = 2048;  // segment starts kept in shared memory up to this many segments

// Stable segmented partition in one pass per stage.  List A is cut into
// segments; within segment k the entries with flag 0 (side[point] == 0) keep
// their order at the front and the flag-1 entries keep their order after the
// segment's nzero[k] zeros.  The destination of entry i needs the number of
// flag-1 entries before i inside its segment = (flag-1 entries before i in
// the whole list) - obefore[k]; the first term comes from a block scan and a
// decoupled look-back over the preceding tiles (tiles in ticket order,
// bounded waits).  The flags of the NEXT stage, which cuts the list written
// here, follow from each entry's destination and are written on the way.
// Tile status words: bits 62-63 = 0 (not yet), 1 (aggregate), 2 (inclusive
// prefix); [0, T) tiles, [T] ticket; zeroed before every stage.
__global__ void __launch_bounds__(kPartThreads) k_part_fused(
    const int32_t* __restrict__ A, const uint8_t* __restrict__ side, int n, const int32_t* __restrict__ start,
    const int32_t* __restrict__ nzero, const int32_t* __restrict__ obefore, int K, int32_t* __restrict__ out,
    const int32_t* __restrict__ nstart, const int32_t* __restrict__ nnzero, int nK, uint8_t* __restrict__ side_next,
    int direct_next, unsigned long long* tstat, int T, unsigned* status, GeomArgs geo) {
    pdl_wait();
    __shared__ int wsum[32];
    __shared__ int sh_tile;
    __shared__ long long sh_excl;
    __shared__ int32_t s_start[kPartSegSmem + 1];  // the segment starts, when they fit
    const bool seg_smem = K <= kPartSegSmem;
    if (seg_smem)
        for (int q = threadIdx.x; q <= K; q += kPartThreads) s_start[q] = start[q];
    __syncthreads();
    const int32_t* segs = seg_smem ? s_start : start;
    unsigned long long* ticket = tstat + T;
    while (true) {
        if (threadIdx.x == 0) sh_tile = (int)atomicAdd(ticket, 1ull);
        __syncthreads();
        const int t = sh_tile;  // rewritten only after the scan's barriers of this tile
        if (t >= T) break;
        const int i0 = t * kPartTile + threadIdx.x * kPartItems;
        int f[kPartItems], a[kPartItems];
        int sum = 0;
#pragma unroll
        for (int j = 0; j < kPartItems; ++j) {
            const int i = i0 + j;
            a[j] = i < n ? A[i] : 0;
            f[j] = i < n ? (int)side[a[j]] : 0;
            sum += f[j];
        }
        int total;
        const int excl = block_excl_scan_nb(sum, wsum, total);  // the barrier after the look-back closes it
        if (threadIdx.x < 32) {
            const unsigned long long pre = warp_lookback(tstat, t, (unsigned long long)total, status);
            if (threadIdx.x == 0) sh_excl = (long long)pre;
        }
        __syncthreads();
        if (i0 >= n) continue;
        long long P = sh_excl + excl;  // flag-1 entries before position i0
        int k = find_seg_any(segs, K, i0);
        int s = segs[k], e = segs[k + 1], nz = nzero[k];
        long long ob = obefore[k];
#pragma unroll
        for (int j = 0; j < kPartItems; ++j) {
            const int i = i0 + j;
            if (i >= n) break;
            while (i >= e) {
                ++k;
                s = segs[k];
                e = segs[k + 1];
                nz = nzero[k];
                ob = obefore[k];
            }
            const int ones = (int)(P - ob);
            const int dst = f[j] ? s + nz + ones : i - ones;
            if (dst >= s && dst < e) {
                out[dst] = a[j];
                if (side_next) {
                    // one tree: segment k's side-f part is segment 2k + f of the next stage (a box's halves,
                    // a half box's bottom / top); a forest's finished instances keep one segment: search
                    const int kn = direct_next ? 2 * k + f[j] : find_seg(nstart, nK, dst);
                    side_next[a[j]] = (uint8_t)((dst - nstart[kn]) >= nnzero[kn]);
                }
            } else {
                atomicOr(status, ST_INTERNAL);
            }
            P += f[j];
        }
    }
    // the geometry of the level whose lists this stage reads (none: geo.cnt = 0), after the tiles, so that no
    // tile waits on it; it takes the place of a launch between the stages
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < geo.cnt; q += gridDim.x * blockDim.x) geom_box(geo, q);
}

// One stage: partition A by side (segments of `seg`) into out; with `next`,
// also the flags of the next stage's cut of out.
// Stage `stage` uses its own region of tile status words (T + 1 each, zeroed
// together before the first stage of a build).
// geo: the geometry the stage's CTAs compute after their tiles (geo.cnt = 0: none).
static fmm_status partition(Tree& t, cudaStream_t s, int stage, const int32_t* A, const uint8_t* side,
                            const SegTable& seg, int32_t* out, const SegTable* next, uint8_t* side_next,
                            const GeomArgs& geo) {
    const int n = (int)t.n;
    const int T = nblk(n, kPartTile);
    const int grid = std::min(T, t.num_sms * 8);  // a CTA per tile up to 8 per SM: more warps to hide the load chain
    launch_dep(true, k_part_fused, grid, kPartThreads, 0, s,
               A, side, n, seg.d_start, seg.d_nzero, seg.d_obefore, seg.K, out, next ? next->d_start : nullptr,
               next ? next->d_nzero : nullptr, next ? next->K : 0, next ? side_next : nullptr, t.ninst == 1 ? 1 : 0,
               t.d_part_stat + (size_t)stage * (T + 1), T, t.d_status, geo);
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

// One thread per box of a level whose geometry no partition stage carries.
__global__ void k_geom(GeomArgs g) {
    pdl_wait();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < g.cnt) geom_box(g, q);
}

// ============================================== subtree splits in one CTA
//
// From level l0 on every box holds at most kSubMax points, so one CTA takes a
// box of level l0 and performs all of its remaining median splits in shared
// memory: the x- and y-lists become arrays of 16-bit local ids (local id =
// position in the box's x-list), the side flags live in shared memory, and
// each stable partition is a block-wide scan.  Geometry of every new box is
// computed on the way; at the end the box's leaf-ordered list of input
// indices is written back over its part of the global y-list.

constexpr int kSubThreads = 1024;  // measured: 1024 beats 256 and 512 (rebuild 1.156 -> 1.132 ms)
constexpr int kSubItems = kSubMax / kSubThreads;
constexpr int kSubSegs = 2048;       // segments (half boxes) per split stage

__device__ __forceinline__ void box_geometry(int b, double x0, double x1, double y0, double y1,
                                             const double2* __restrict__ center_root_src, int root,
                                             double2* center, double* radius, double* rho, float4* chl,
                                             float* rho32, float* rad32) {
    const double cx = __dmul_rn(0.5, __dadd_rn(x0, x1));
    const double cy = __dmul_rn(0.5, __dadd_rn(y0, y1));
    const double dx = __dsub_rn(x1, x0), dy = __dsub_rn(y1, y0);
    const double r = __dmul_rn(0.5, __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))));
    center[b] = make_double2(cx, cy);
    radius[b] = r;
    rad32[b] = __double2float_rn(r);
    double ox = cx, oy = cy, rfloor = 0.0;
    if (root >= 0) {
        const double2 o = center_root_src[root];
        ox = o.x;
        oy = o.y;
        rfloor = ldexp(radius[root], -24);
    }
    const double rs = r > rfloor ? r : rfloor;
    const float r32 = rs >= 1e-30 ? __double2float_rn(rs) : 0.0f;
    rho32[b] = r32;
    rho[b] = (double)r32;
    const double ex = __dsub_rn(cx, ox), ey = __dsub_rn(cy, oy);
    const float hx = __double2float_rn(ex), hy = __double2float_rn(ey);
    chl[b] = make_float4(hx, hy, __double2float_rn(__dsub_rn(ex, (double)hx)),
                         __double2float_rn(__dsub_rn(ey, (double)hy)));
}

// Stable partition of lin (n local ids) within segments st[0..nseg): code[id]
// = 2 * (segment of id) + side of id; segment k keeps its side-0 entries
// first (the first nz[k] positions), both sides in their input order.  A thread
// keeps the running prefix of side-1 entries of its own positions in
// registers; segpre[k] receives the prefix at segment k's first position.
__device__ __forceinline__ void cta_partition(const uint16_t* lin, uint16_t* lout, int n, const uint16_t* st,
                                              const uint16_t* nz, const uint16_t* code, uint16_t* segpre,
                                              int* wsum) {
    const int i0 = threadIdx.x * kSubItems;
    int c[kSubItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kSubItems; ++k) {
        const int i = i0 + k;
        c[k] = i < n ? code[lin[i]] : 0;
        sum += c[k] & 1;
    }
    int total;
    int acc = block_excl_scan(sum, wsum, total);
    int pre[kSubItems];
#pragma unroll
    for (int k = 0; k < kSubItems; ++k) {
        pre[k] = acc;
        if (i0 + k < n && st[c[k] >> 1] == i0 + k) segpre[c[k] >> 1] = (uint16_t)acc;
        acc += c[k] & 1;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSubItems; ++k) {
        const int i = i0 + k;
        if (i >= n) break;
        const int sgi = c[k] >> 1;
        const int s0 = st[sgi];
        const int ones = pre[k] - (int)segpre[sgi];
        const int dst = (c[k] & 1) ? s0 + nz[sgi] + ones : s0 + (i - s0) - ones;
        if (dst >= 0 && dst < n) lout[dst] = lin[i];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSubThreads) k_subtree(
    const int32_t* __restrict__ ids, int cnt, int l0, const int32_t* __restrict__ X, int32_t* __restrict__ Y,
    const double2* __restrict__ xy, const int32_t* __restrict__ bstart, const int32_t* __restrict__ bcount,
    const int32_t* __restrict__ inst, const int64_t* __restrict__ inst_box_off, const int32_t* __restrict__ inst_levels,
    int32_t* __restrict__ loc, double2* center, double* radius, double* rho, float4* chl, float* rho32, float* rad32,
    unsigned* status) {
    pdl_wait();
    __shared__ uint16_t buf[3][kSubMax];
    // per local id: its box (then half box) numbered within the subtree level, and during a split
    // 2 * that + the side it goes to
    __shared__ uint16_t bid[kSubMax];
    __shared__ uint16_t st[kSubSegs], nz[kSubSegs], segpre[kSubSegs];
    __shared__ int wsum[32];
    if (blockIdx.x >= cnt) return;
    const int B = ids[blockIdx.x];
    const int s = bstart[B], n = bcount[B];
    if (n > kSubMax) {  // the host picks l0 so that this cannot happen
        if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
        return;
    }
    const int ib = inst[B];
    const int bo = (int)inst_box_off[ib];
    const int Lb = inst_levels[ib];
    long long off_l0 = 0, w = 1;
    for (int q = 0; q < l0; ++q) {
        off_l0 += w;
        w *= 4;
    }
    const int iB = B - bo - (int)off_l0;
    uint16_t* xl = buf[0];  // local ids in x-order within the current boxes
    uint16_t* yl = buf[1];  // local ids in y-order within the current boxes
    uint16_t* tp = buf[2];
    for (int i = threadIdx.x; i < n; i += kSubThreads) {
        loc[X[s + i]] = i;
        xl[i] = (uint16_t)i;
        bid[i] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSubThreads) yl[i] = (uint16_t)loc[Y[s + i]];
    __syncthreads();
    long long off_l = off_l0, width = 1, lsz = w;  // level offset, subtree boxes and all boxes on level l
    for (int l = l0; l + 1 < Lb; ++l) {
        const int gb0 = bo + (int)off_l + iB * (int)width;  // first box of the subtree on level l
        if (2 * width > kSubSegs) {  // cannot happen for boxes of <= kSubMax non-empty leaves
            if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
            return;
        }
        // x-split: segments = boxes of level l
        for (int k = threadIdx.x; k < width; k += kSubThreads) {
            st[k] = (uint16_t)(bstart[gb0 + k] - s);
            nz[k] = (uint16_t)(bcount[gb0 + k] / 2);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kSubThreads) {
            const int id = xl[i];
            const int k = bid[id];
            bid[id] = (uint16_t)(2 * k + ((i - st[k]) >= nz[k]));  // box k's left / right half: 2k / 2k+1
        }
        __syncthreads();
        cta_partition(yl, tp, n, st, nz, bid, segpre, wsum);  // tp = new y-list
        // y-split of every half: segments = half boxes
        for (int k = threadIdx.x; k < width; k += kSubThreads) {
            const int bs = bstart[gb0 + k] - s, bn = bcount[gb0 + k], nl = bn / 2;
            st[2 * k] = (uint16_t)bs;
            st[2 * k + 1] = (uint16_t)(bs + nl);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < width; k += kSubThreads) {
            const int bn = bcount[gb0 + k], nl = bn / 2;
            nz[2 * k] = (uint16_t)(nl / 2);
            nz[2 * k + 1] = (uint16_t)((bn - nl) / 2);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kSubThreads) {
            const int id = tp[i];
            const int k = bid[id];
            // half box k's bottom / top: 2k / 2k+1 = 4 (box) + 2 (x side) + (y side), the order lb, lt, rb, rt
            bid[id] = (uint16_t)(2 * k + ((i - st[k]) >= nz[k]));
        }
        __syncthreads();
        cta_partition(xl, yl, n, st, nz, bid, segpre, wsum);  // old y-list buffer = new x-list
        {
            uint16_t* nx = yl;
            uint16_t* ny = tp;
            tp = xl;
            xl = nx;
            yl = ny;
        }
        off_l += lsz;  // first box of level l+1
        lsz *= 4;
        width *= 4;
        // geometry of the children (level l+1)
        const int gc0 = bo + (int)off_l + iB * (int)width;
        for (int k = threadIdx.x; k < width; k += kSubThreads) {
            const int b = gc0 + k;
            const int cs = bstart[b] - s, ce = cs + bcount[b] - 1;
            const double x0 = xy[X[s + xl[cs]]].x, x1 = xy[X[s + xl[ce]]].x;
            const double y0 = xy[X[s + yl[cs]]].y, y1 = xy[X[s + yl[ce]]].y;
            box_geometry(b, x0, x1, y0, y1, center, bo, center, radius, rho, chl, rho32, rad32);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += kSubThreads) Y[s + i] = X[s + yl[i]];
}

// Separate evaluation points (the tree holds n_src sources, then the evaluation
// points): one warp per leaf places the leaf's sources first in its slot
// block, in sorted order, and its evaluation points after them, and records
// the leaf's source count.  Y = input index of every sorted position.
__global__ void k_target_slots(const int32_t* __restrict__ leaves, int nleaf, const int32_t* __restrict__ bstart,
                               const int32_t* __restrict__ bcount, const int32_t* __restrict__ pslot,
                               const int32_t* __restrict__ Y, int n_src, int32_t* __restrict__ slot_of,
                               int32_t* __restrict__ nsrc) {
    pdl_wait();
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nleaf) return;  // warp-uniform
    const int b = leaves[w];
    const int s = bstart[b], c = bcount[b], ps = pslot[b];
    int ns = 0;
    for (int i0 = 0; i0 < c; i0 += 32) {
        const bool src = i0 + lane < c && Y[s + i0 + lane] < n_src;
        ns += __popc(__ballot_sync(0xffffffffu, src));
    }
    int before_s = 0, before_t = 0;
    for (int i0 = 0; i0 < c; i0 += 32) {
        const bool in = i0 + lane < c;
        const bool src = in && Y[s + i0 + lane] < n_src;
        const unsigned ms = __ballot_sync(0xffffffffu, src), mt = __ballot_sync(0xffffffffu, in && !src);
        const unsigned below = (1u << lane) - 1u;
        if (in)
            slot_of[s + i0 + lane] = ps + (src ? before_s + __popc(ms & below) : ns + before_t + __popc(mt & below));
        before_s += __popc(ms);
        before_t += __popc(mt);
    }
    if (lane == 0) nsrc[b] = ns;
}

// Sorted point data: permutation, FP64 copy, FP32 hi/lo split relative to the
// instance origin (root centre), and the leaf of every sorted position.
// The P2P operands also go to the leaf slot layout: leaf q's points fill slots
// q*cap, q*cap+1, ...  FP64 path: the point per slot.  FP32 path: slots are
// interleaved in pairs (2m, 2m+1) for packed f32x2 arithmetic, as two float4
// (x_hi[2m], x_hi[2m+1], y_hi[2m], y_hi[2m+1]), (x_lo.., x_lo.., y_lo.., y_lo..).
__global__ void k_finalize(const int32_t* __restrict__ Y, int n, const double2* __restrict__ xy,
                           const int32_t* __restrict__ inst, const int64_t* __restrict__ inst_box_off,
                           const double2* __restrict__ center, int32_t* perm, double2* pts, float4* pos4,
                           const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ slot_of, float* posp32,
                           double2* posp64) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int id = Y[i];
    perm[i] = id;
    const double2 p = xy[id];
    pts[i] = p;
    const int lf = leaf_of[i];      // leaf and slot of a sorted position follow from the shape alone
    const int slot = slot_of[i];
    const double2 o = center[inst_box_off[inst[lf]]];
    const double ex = __dsub_rn(p.x, o.x), ey = __dsub_rn(p.y, o.y);
    const float hx = __double2float_rn(ex), hy = __double2float_rn(ey);
    const float4 v = make_float4(hx, hy, __double2float_rn(__dsub_rn(ex, (double)hx)),
                                 __double2float_rn(__dsub_rn(ey, (double)hy)));
    pos4[i] = v;
    if (posp32) {
        float* f = posp32 + 8 * (slot >> 1) + (slot & 1);
        f[0] = v.x;
        f[2] = v.y;
        f[4] = v.z;
        f[6] = v.w;
    }
    if (posp64) posp64[slot] = p;
}

// ================================================================== lists
//
// Level by level.  The candidates of level l are the pairs (child c of parent
// P, child c' of the j-th strong entry Q of P), enumerated as
//     g = 16*(soff(P) - base(l-1)) + c*4*ns(P) + 4*j + c'
// so that the candidates of one child box are contiguous and in (j, c')
// order.  Every candidate is classified (strong / weak / none, the last for
// entries of boxes without children), the flags are scanned over tiles, and a
// scatter writes the lists in candidate order.  The strong entries of level l
// are stored contiguously after those of level l-1; `owner` records the box of
// every strong entry, which decodes the next level's candidates.

__global__ void k_lists_root(const int64_t* __restrict__ inst_box_off, int ninst, int32_t* soff, int32_t* ns,
                             int32_t* sidx, int32_t* sowner, int32_t* woff, int32_t* nw,
                             unsigned long long* lvl_base, const int32_t* __restrict__ child0,
                             const int32_t* __restrict__ pslot, const int32_t* __restrict__ bcount, int2* srng) {
    pdl_wait();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) {
        lvl_base[0] = 0;             // strong entries of level 0 start at 0
        lvl_base[1] = ninst;         // ... and level 1 after them
        lvl_base[kMaxLevels + 0] = 0;  // weak entries
        lvl_base[kMaxLevels + 1] = 0;
    }
    if (b >= ninst) return;
    const int r = (int)inst_box_off[b];
    soff[r] = b;
    ns[r] = b + 1;  // list ends (lengths are end - first entry)
    sidx[b] = r;
    sowner[b] = r;
    woff[r] = 0;
    nw[r] = 0;
    if (child0[r] < 0) srng[b] = make_int2(pslot[r], bcount[r]);  // a one-level instance: its P2P sources
}

// eq (2.3) in FP64: R + theta*r <= theta*d, with d > 0 required.
__device__ __forceinline__ bool well_separated(double2 ca, double ra, double2 cb, double rb, double theta) {
    const double dx = __dsub_rn(ca.x, cb.x), dy = __dsub_rn(ca.y, cb.y);
    const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    const double R = ra > rb ? ra : rb;
    const double r = ra > rb ? rb : ra;
    return d > 0.0 && __dadd_rn(R, __dmul_rn(theta, r)) <= __dmul_rn(theta, d);
}

// The exact FP64 test for pairs the FP32 test cannot decide (out of line:
// rare, and it keeps the FP64 code off the classification path).
__device__ __noinline__ bool well_separated_exact(int a, int b, const double2* __restrict__ center,
                                                 const double* __restrict__ radius, double theta) {
    return well_separated(center[a], radius[a], center[b], radius[b], theta);
}

// Same decision, evaluated in FP32 first on squared quantities:
// (R + theta r)^2 against theta^2 |ca - cb|^2 with the centres as hi/lo pairs
// (so the difference keeps FP32 relative accuracy) and the radii as floats;
// only pairs within a relative 4e-5 of the boundary (far above the FP32
// evaluation error) repeat the exact FP64 test, so the result equals the FP64
// test bit for bit.  ca / ra: box a's centre and radius, already loaded.
__device__ __forceinline__ bool well_separated_fast(int a, const float4 ca, float ra, int b,
                                                    const float4* __restrict__ chl, const float* __restrict__ rad32,
                                                    const double2* __restrict__ center,
                                                    const double* __restrict__ radius, float theta32, double theta) {
    const float4 cb = chl[b];
    const float rb = rad32[b];
    const float dx = (ca.x - cb.x) + (ca.z - cb.z);
    const float dy = (ca.y - cb.y) + (ca.w - cb.w);
    const float lhs = fmaf(theta32, fminf(ra, rb), fmaxf(ra, rb));
    const float l2 = lhs * lhs;
    const float r2 = (theta32 * theta32) * fmaf(dx, dx, dy * dy);
    const float tol = 4e-5f * (l2 + r2);
    if (l2 + tol < r2) return true;
    if (l2 > r2 + tol) return false;
    return well_separated_exact(a, b, center, radius, theta);
}

// The four candidates g = 4*q + c' (c' = 0..3) share the child box b and the
// strong entry Q of its parent; decode that group once.
struct CandGroup {
    int b, h0;      // child box, first child of Q (candidates h0 + c')
    bool first;     // group holds the first candidate of b
    bool last;      // group holds the last candidate of b
    bool valid;     // the parent has children
};

__device__ __forceinline__ CandGroup decode_group(long long q, long long base_prev, const int32_t* __restrict__ sowner,
                                                  const int32_t* __restrict__ soff, const int32_t* __restrict__ ns,
                                                  const int32_t* __restrict__ sidx,
                                                  const int32_t* __restrict__ child0) {
    CandGroup c;
    const int P = sowner[base_prev + (q >> 2)];
    const int c0 = child0[P];
    c.valid = c0 >= 0;
    if (!c.valid) {
        c.b = c.h0 = 0;
        c.first = c.last = false;
        return c;
    }
    const int n = ns[P] - soff[P];
    const long long e0 = (long long)soff[P] - base_prev;
    const int r = (int)(q - 4 * e0);  // (child index) * n + j
    const int ci = r / n, j = r - ci * n;
    c.b = c0 + ci;
    c.h0 = child0[sidx[soff[P] + j]];
    c.first = j == 0;
    c.last = j == n - 1;
    return c;
}

// 8 candidates per thread: measured equal to 12 and faster than 16
constexpr int kLThreads = 256, kLItems = 8, kLTile = kLThreads * kLItems;

// One pass per level: every candidate is classified (none / strong / weak),
// the tile's strong and weak counts are scanned across the block, the tile's
// offsets come from a decoupled look-back over the preceding tiles, and the
// entries are written in candidate order.  Tiles are taken in ticket order
// (atomic counter), so a tile only waits on tiles that running CTAs already
// hold; every wait is bounded and a timeout is reported as ST_TIMEOUT.
// Tile status words: bits 62-63 = 0 (not yet), 1 (tile aggregate), 2 (inclusive
// prefix); bits 0-61 = the count.  [0, tiles_cap) strong, [tiles_cap, 2
// tiles_cap) weak, then the ticket counter; zeroed before every level.
__global__ void __launch_bounds__(kLThreads) k_lists_level(
    int l, unsigned long long* lvl_base, int32_t* __restrict__ sowner, int32_t* __restrict__ soff,
    int32_t* __restrict__ ns, int32_t* __restrict__ sidx, int32_t* __restrict__ woff, int32_t* __restrict__ nw,
    int32_t* __restrict__ widx, const int32_t* __restrict__ child0, const int32_t* __restrict__ pslot,
    const int32_t* __restrict__ bcount, int2* __restrict__ srng, const float4* __restrict__ chl,
    const float* __restrict__ rad32, const double2* __restrict__ center, const double* __restrict__ radius,
    double theta, unsigned long long* tstat, long long tiles_cap, long long scap, long long wcap,
    unsigned long long* need, unsigned* status) {
    pdl_wait();
    __shared__ int ws[32];
    __shared__ long long sh_excl[2];
    __shared__ long long sh_tile;
    if (*((volatile unsigned*)status) & (ST_STRONG_OVERFLOW | ST_WEAK_OVERFLOW)) return;
    const long long base_prev = (long long)lvl_base[l - 1];
    const long long bs = (long long)lvl_base[l], bw = (long long)lvl_base[kMaxLevels + l];
    const long long ncand = 16 * (bs - base_prev);
    const long long ntiles = (ncand + kLTile - 1) / kLTile;
    if (ntiles > tiles_cap) {  // tile status array too small: grow the candidate capacity
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicMax(need + 0, (unsigned long long)ncand);
            atomicOr(status, ST_STRONG_OVERFLOW);
        }
        return;
    }
    if (ntiles == 0) {  // no candidates: the level's lists are empty
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            lvl_base[l + 1] = (unsigned long long)bs;
            lvl_base[kMaxLevels + l + 1] = (unsigned long long)bw;
        }
        return;
    }
    unsigned long long* ticket = tstat + 2 * tiles_cap;
    const float th32 = (float)theta;
    while (true) {
        if (threadIdx.x == 0) sh_tile = (long long)atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long t = sh_tile;  // rewritten only after the scan's barriers of this tile
        if (t >= ntiles) break;
        const long long g0 = t * kLTile + (long long)threadIdx.x * kLItems;
        CandGroup cg[kLItems / 4];
        uint32_t fl = 0;  // 2 bits per candidate: 0 none, 1 strong, 2 weak
        int cs = 0, cw = 0;
#pragma unroll
        for (int gq = 0; gq < kLItems / 4; ++gq) {
            const long long gg = g0 + 4 * gq;
            cg[gq].valid = false;
            if (gg >= ncand) continue;
            cg[gq] = decode_group(gg >> 2, base_prev, sowner, soff, ns, sidx, child0);
            if (!cg[gq].valid) continue;
            const float4 cb = chl[cg[gq].b];  // the child box, shared by the group's four candidates
            const float rb = rad32[cg[gq].b];
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) {
                const int h = cg[gq].h0 + cp;
                const bool sep = (h != cg[gq].b) &&
                                 well_separated_fast(cg[gq].b, cb, rb, h, chl, rad32, center, radius, th32, theta);
                cs += !sep;
                cw += sep;
                fl |= (sep ? 2u : 1u) << (2 * (4 * gq + cp));
            }
        }
        // both counts in one scan (at most 8 per thread and kLTile per tile: 16 bits each)
        int tot;
        const int pk = block_excl_scan_nb(cs | (cw << 16), ws, tot);
        const int tot_s = tot & 0xffff, tot_w = tot >> 16;
        long long ps = pk & 0xffff;
        long long pw = pk >> 16;
        if (threadIdx.x < 64) {  // warp 0: strong counts, warp 1: weak counts
            const int which = threadIdx.x >> 5;
            const unsigned long long agg = (unsigned long long)(which ? tot_w : tot_s);
            const unsigned long long excl = warp_lookback(tstat + which * tiles_cap, t, agg, status);
            if ((threadIdx.x & 31) == 0) {
                sh_excl[which] = (long long)excl;
                if (t == ntiles - 1) {  // level totals and capacity checks
                    const long long base = which ? bw : bs;
                    const long long end = base + (long long)(excl + agg);
                    lvl_base[which ? kMaxLevels + l + 1 : l + 1] = (unsigned long long)end;
                    if (end > (which ? wcap : scap)) {
                        atomicMax(need + 1 + which, (unsigned long long)end);
                        atomicOr(status, which ? ST_WEAK_OVERFLOW : ST_STRONG_OVERFLOW);
                    }
                }
            }
        }
        __syncthreads();
        ps += sh_excl[0];
        pw += sh_excl[1];
#pragma unroll
        for (int gq = 0; gq < kLItems / 4; ++gq) {
            const CandGroup& c = cg[gq];
            if (!c.valid) continue;
            if (c.first) {
                soff[c.b] = (int32_t)(bs + ps);
                woff[c.b] = (int32_t)(bw + pw);
            }
            const bool leaf = child0[c.b] < 0;
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) {
                const int h = c.h0 + cp;
                if (((fl >> (2 * (4 * gq + cp))) & 3u) == 1u) {
                    const long long qq = bs + ps;
                    if (qq < scap) {
                        sidx[qq] = h;
                        sowner[qq] = c.b;
                        if (leaf) srng[qq] = make_int2(pslot[h], bcount[h]);
                    }
                    ++ps;
                } else {
                    if (bw + pw < wcap) widx[bw + pw] = h;
                    ++pw;
                }
            }
            if (c.last) {
                ns[c.b] = (int32_t)(bs + ps);  // list end
                nw[c.b] = (int32_t)(bw + pw);
            }
        }
    }
}

// Work items that bound the work of one warp / thread whatever the list
// lengths: P2P items = (leaf, slice of its strong list) with about
// p2p_item_sources(n) source points, M2L items = (box, at most m2l_item_pairs() weak
// entries).  A box whose list is split keeps its items contiguous; their
// partial sums are added in item order later (deterministic).
// int4 item = (box, list begin, list end, first item of the box or -1 when
// the box has a single item).
// One atomic per block and counter: the block's threads reserve k[q] entries
// from the global counters c[q] (q < 5; a zero block total issues no atomic)
// and get their first entries in b[q], in thread order.  Two block barriers.
__device__ __forceinline__ void block_reserve5(unsigned long long* const (&c)[5], const int (&k)[5],
                                               unsigned long long (&b)[5]) {
    __shared__ int wtot[5][32];
    __shared__ unsigned long long base[5];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) incl[q] = k[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int y = __shfl_up_sync(0xffffffffu, incl[q], o);
            if (lane >= o) incl[q] += y;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < 5; ++q) wtot[q][w] = incl[q];
    }
    __syncthreads();
    if (w == 0) {
        int tot[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            int v = lane < nw ? wtot[q][lane] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < nw) wtot[q][lane] = x - v;  // warps before this one
            tot[q] = __shfl_sync(0xffffffffu, x, 31);
        }
        // lanes 0-4 issue the block's atomics side by side
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (lane == q) base[q] = tot[q] > 0 ? atomicAdd(c[q], (unsigned long long)tot[q]) : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 5; ++q) b[q] = base[q] + (unsigned long long)(wtot[q][w] + incl[q] - k[q]);
}

// M2L rows (the order in which the M2L kernels take the items): a box's full
// items (K pairs) take consecutive rows from rowctr[kM2LItemPairsMax]; its
// short last item (length r < K) is counted in rowctr[r] and placed by
// k_m2l_rows once all counts are known.
__global__ void k_items(int nbox, const int32_t* __restrict__ child0, const int32_t* __restrict__ bcount,
                        const int32_t* __restrict__ soff, const int32_t* __restrict__ ns,
                        const int32_t* __restrict__ woff, const int32_t* __restrict__ nw, unsigned long long* ctr,
                        int4* p2p_items, int32_t* p2p_rows, int2* leaf_items, long long p2p_cap, int4* m2l_items,
                        int2* box_m2l,
                        long long m2l_cap, int K, unsigned long long* rowctr, int32_t* rows, int2* box_tail,
                        unsigned* status, int item_sources) {
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    // lists that overflowed or whose build gave up: no items (the counters stay zero)
    if (*((volatile unsigned*)status) & (ST_STRONG_OVERFLOW | ST_WEAK_OVERFLOW | ST_TIMEOUT | ST_INTERNAL)) return;
    const bool in = b < nbox;
    const bool leaf = in && child0[b] < 0;
    int kp = 0, C = 1, n = 0;
    if (leaf) {
        n = ns[b] - soff[b];
        C = max(1, item_sources / max(bcount[b], 1));
        kp = (n + C - 1) / C;
    }
    const int m = in ? nw[b] - woff[b] : 0;
    const int km = (m + K - 1) / K;
    const int nfull = m / K, r = m - nfull * K;
    const int rank = r > 0 ? (int)atomicAdd(rowctr + r, 1ull) : 0;  // issued first: its latency overlaps the rest
    // P2P row order: the full items of split leaves (the heavy ones) take rows from the front, every leaf's
    // last (or only) item takes a row from the back of the capacity
    const int kh = kp > 1 ? kp - 1 : 0, kl = kp > 0 ? 1 : 0;
    unsigned long long* const cs[5] = {ctr + 2, ctr + 3, rowctr + kM2LItemPairsMax, rowctr + kM2LItemPairsMax + 1,
                                       rowctr + kM2LItemPairsMax + 2};
    const int ks[5] = {kp, km, nfull, kh, kl};
    unsigned long long bs[5];
    block_reserve5(cs, ks, bs);
    const unsigned long long bp = bs[0], bm = bs[1], bf = bs[2], bh = bs[3], bl = bs[4];
    // a box whose items do not fit gets (0, 0): the passes that read these tables stay inside the buffers
    if (leaf) {
        if ((long long)(bp + kp) > p2p_cap || (long long)(bh + kh + bl + kl) > p2p_cap) {
            leaf_items[b] = make_int2(0, 0);
            atomicOr(status, ST_ITEM_OVERFLOW);
        } else {
            leaf_items[b] = make_int2((int)bp, kp);
            for (int c = 0; c < kp; ++c)
                p2p_items[bp + c] = make_int4(b, c * C, min(n, (c + 1) * C), kp > 1 ? (int)bp : -1);
            for (int c = 0; c < kh; ++c) p2p_rows[bh + c] = (int32_t)(bp + c);
            if (kl) p2p_rows[p2p_cap - 1 - (long long)bl] = (int32_t)(bp + kp - 1);
        }
    }
    if (!in) return;
    box_tail[b] = make_int2(r, rank);
    if ((long long)(bm + km) > m2l_cap) {
        box_m2l[b] = make_int2(0, 0);
        atomicOr(status, ST_ITEM_OVERFLOW);
    } else {
        box_m2l[b] = make_int2((int)bm, km);
        for (int c = 0; c < km; ++c)
            m2l_items[bm + c] = make_int4(b, c * K, min(m, (c + 1) * K), km > 1 ? (int)bm : -1);
        for (int c = 0; c < nfull; ++c) {
            if ((long long)(bf + c) < m2l_cap) rows[bf + c] = (int32_t)(bm + c);
            else atomicOr(status, ST_ITEM_OVERFLOW);
        }
    }
}

// Rows of the short last items: after the full items, by decreasing length
// (rank among equal lengths from k_items' counter).  Blocks of kM2LItemPairsMax threads.
static_assert(kM2LItemPairsMax == 256, "k_m2l_rows: one thread per item length in its blocks of 256");
// After an item overflow the P2P and M2L item counts move to need[4], need[5] (the sizes the host grows the
// capacities to) and the counters read by the evaluation are zeroed, so that an evaluation already queued
// behind this build finds no items.
__global__ void k_m2l_rows(int nbox, const int2* __restrict__ box_m2l, const int2* __restrict__ box_tail,
                           const unsigned long long* __restrict__ rowctr, long long m2l_cap, int32_t* rows,
                           unsigned long long* item_ctr, unsigned long long* need, unsigned* status) {
    pdl_wait();
    __shared__ unsigned long long base[kM2LItemPairsMax];
    __shared__ int wsum[32];
    const unsigned st0 = *((volatile unsigned*)status);
    if ((st0 & ST_ITEM_OVERFLOW) && blockIdx.x == 0 && threadIdx.x == 0) {
        need[4] = item_ctr[0];
        need[5] = item_ctr[1];
        item_ctr[0] = 0;
        item_ctr[1] = 0;
    }
    if (st0 & (ST_STRONG_OVERFLOW | ST_WEAK_OVERFLOW | ST_ITEM_OVERFLOW | ST_TIMEOUT)) return;  // uniform
    {  // base[r] = full items + short items longer than r: thread i takes length r = kM2LItemPairsMax - 1 - i
        const int r = kM2LItemPairsMax - 1 - (int)threadIdx.x;
        const int c = r >= 1 ? (int)rowctr[r] : 0;
        int total;
        const int ex = block_excl_scan(c, wsum, total);
        if (r >= 0) base[r] = rowctr[kM2LItemPairsMax] + (unsigned long long)ex;
    }
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int2 tl = box_tail[b];
    if (tl.x <= 0) return;
    const int2 mi = box_m2l[b];
    const unsigned long long pos = base[tl.x] + (unsigned long long)tl.y;
    if ((long long)pos < m2l_cap) rows[pos] = mi.x + mi.y - 1;
    else atomicOr(status, ST_INTERNAL);
}

// Totals for fmm_get_tree_info (diagnostics, not on the evaluation path).
__global__ void k_count(const int32_t* __restrict__ leaf_ids, int nleaf, const int32_t* __restrict__ soff,
                        const int32_t* __restrict__ ns, const int32_t* __restrict__ sidx,
                        const int32_t* __restrict__ bcount, unsigned long long* out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long sl = 0, pp = 0;
    if (q < nleaf) {
        const int b = leaf_ids[q];
        const int n = ns[b] - soff[b];
        sl = n;
        unsigned long long src = 0;
        for (int j = 0; j < n; ++j) src += bcount[sidx[soff[b] + j]];
        pp = src * (unsigned long long)bcount[b];
    }
    for (int o = 16; o; o >>= 1) {
        sl += __shfl_xor_sync(0xffffffffu, sl, o);
        pp += __shfl_xor_sync(0xffffffffu, pp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (sl) atomicAdd(out + 0, sl);
        if (pp) atomicAdd(out + 1, pp);
    }
}

// ============================================================ orchestration

static void dfree(void* p) {
    if (p) cudaFree(p);
}

template <typename T>
static fmm_status dalloc(T** p, size_t count) {
    dfree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error("device allocation failed");
        return FMM_ERR_OOM;
    }
    FMM_CUDA(e);
    return FMM_OK;
}

fmm_status alloc_build(Tree& t) {
    const size_t n = (size_t)t.n;
    fmm_status st;
    for (int i = 0; i < 4; ++i) {
        if ((st = dalloc(&t.d_keys[i], n))) return st;
        if ((st = dalloc(&t.d_vals[i], n))) return st;
    }
    if ((st = dalloc(&t.d_X2, n))) return st;
    if ((st = dalloc(&t.d_Y2, n))) return st;
    if ((st = dalloc(&t.d_sideX, n))) return st;
    if ((st = dalloc(&t.d_sideY, n))) return st;
    if ((st = dalloc(&t.d_loc, n))) return st;
    const int64_t T = std::max<int64_t>(nblk(t.n, kPartTile), nblk(t.n, kSortTile));
    if ((st = dalloc(&t.d_part_stat, (T + 1) * (size_t)std::max(2 * (t.Lmax - 1), 1)))) return st;  // one region per stage
    if ((st = dalloc(&t.d_sort_hist, 2 * 256 * (size_t)T))) return st;
    if ((st = dalloc(&t.d_sort_off, 2 * 256 * (size_t)T))) return st;
    if ((st = dalloc(&t.d_sort_tot, 2 * 256))) return st;
    if ((st = dalloc(&t.d_sort_os, sort_scratch_words(t.n)))) return st;
    if ((st = dalloc(&t.d_perm, n))) return st;
    if ((st = dalloc(&t.d_pts, n))) return st;
    if ((st = dalloc(&t.d_pos4, n))) return st;
    {
        // leaf (box id) and P2P slot of every sorted position: shape-only, so tabulated once here
        std::vector<int32_t> lo((size_t)t.n), so((size_t)t.n);
        for (int64_t q = 0; q < t.nleaf; ++q) {
            const int32_t b = t.h_leaves[(size_t)q], s0 = t.h_bstart[(size_t)b], c = t.h_bcount[(size_t)b];
            for (int32_t i = 0; i < c; ++i) {
                lo[(size_t)(s0 + i)] = b;
                so[(size_t)(s0 + i)] = (int32_t)(q * t.leaf_cap + i);
            }
        }
        if ((st = upload(&t.d_leaf_of, lo))) return st;
        if ((st = upload(&t.d_slot_of, so))) return st;
    }
    {
        // slot layout (+1 block of padding); padding stays zero across rebuilds of this shape
        const int64_t slots = (t.nleaf + 1) * (int64_t)t.leaf_cap;
        float4* pp = static_cast<float4*>(t.d_posp);
        t.d_posp = nullptr;
        if ((st = dalloc(&pp, (size_t)slots))) return st;
        t.d_posp = pp;
        FMM_CUDA(cudaMemset(t.d_posp, 0, (size_t)slots * sizeof(float4)));
        t.slot_alloc = slots;
    }
    const size_t nb = (size_t)t.nbox;
    if ((st = dalloc(&t.d_center, nb))) return st;
    if ((st = dalloc(&t.d_radius, nb))) return st;
    if ((st = dalloc(&t.d_rho, nb))) return st;
    if ((st = dalloc(&t.d_chl, nb))) return st;
    if ((st = dalloc(&t.d_rho32, nb))) return st;
    if ((st = dalloc(&t.d_rad32, nb))) return st;
    if ((st = dalloc(&t.d_soff, nb))) return st;
    if ((st = dalloc(&t.d_ns, nb))) return st;
    if ((st = dalloc(&t.d_woff, nb))) return st;
    if ((st = dalloc(&t.d_nw, nb))) return st;
    if ((st = dalloc(&t.d_leaf_items, nb))) return st;
    if ((st = dalloc(&t.d_box_m2l, nb))) return st;
    if ((st = dalloc(&t.d_box_tail, nb))) return st;
    if (t.n_src > 0 && (st = dalloc(&t.d_nsrc, nb))) return st;
    // M2L row counters, then the P2P row counters (heavy, light, spare)
    if ((st = dalloc(&t.d_m2l_rowctr, kM2LItemPairsMax + 4))) return st;
    if (!t.d_status) {
        if ((st = dalloc(reinterpret_cast<unsigned long long**>(&t.d_status), 8))) return st;
    }
    if (t.scap_tot < (long long)t.nbox * 16) t.scap_tot = (long long)t.nbox * 16;
    if (t.wcap_tot < (long long)t.nbox * 48) t.wcap_tot = (long long)t.nbox * 48;
    if (t.p2p_cap < t.nleaf * 2) t.p2p_cap = t.nleaf * 2;
    if (t.cand_cap < t.nbox * 64) t.cand_cap = t.nbox * 64;
    if (!t.d_lvl_base) {
        if ((st = dalloc(&t.d_lvl_base, 2 * kMaxLevels + 8))) return st;
    }
    if (t.m2l_cap < t.nbox * 2) t.m2l_cap = t.nbox * 2;
    return alloc_lists(t);
}

fmm_status alloc_lists(Tree& t) {
    fmm_status st;
    if ((st = dalloc(&t.d_sidx, (size_t)t.scap_tot))) return st;
    if ((st = dalloc(&t.d_sowner, (size_t)t.scap_tot))) return st;
    if ((st = dalloc(&t.d_srng, (size_t)t.scap_tot))) return st;
    const size_t tiles = (size_t)(t.cand_cap / kLTile + 2);
    if ((st = dalloc(&t.d_ltstat, (2 * tiles + 1) * (size_t)std::max(t.Lmax - 1, 1)))) return st;  // one region per level
    if ((st = dalloc(&t.d_widx, (size_t)t.wcap_tot))) return st;
    if ((st = dalloc(&t.d_p2p_items, (size_t)t.p2p_cap))) return st;
    if ((st = dalloc(&t.d_p2p_rows, (size_t)t.p2p_cap))) return st;
    if ((st = dalloc(&t.d_m2l_items, (size_t)t.m2l_cap))) return st;
    if ((st = dalloc(&t.d_m2l_rows, (size_t)t.m2l_cap))) return st;
    return FMM_OK;
}

fmm_status run_tree_build(Tree& t, const double* d_xy, cudaStream_t s) {
    const int n = (int)t.n;
    const double2* xy = reinterpret_cast<const double2*>(d_xy);
    FMM_CUDA(cudaMemsetAsync(t.d_status, 0, sizeof(unsigned), s));
    // LSD passes over the 64-bit keys (+2 over the instance index when
    // batched); an even number of passes leaves the result in buffers 0/1.
    int src = 0;
    fmm_status st;
    const int lglob = std::min(t.l0, t.Lmax - 1);  // levels split by the global passes
    // the zeroing comes first, so that the build's kernels follow one another directly (launch_dep)
    if (lglob > 0)
        FMM_CUDA(cudaMemsetAsync(t.d_part_stat, 0,
                                 (size_t)2 * lglob * (nblk(n, kPartTile) + 1) * sizeof(unsigned long long), s));
    bool marked = false;                           // side flags of the first cut already written
    if (n < (1 << 30)) {  // onesweep passes (30-bit counts in the tile status words); keys formed in the first
        // the short sort (high halves + runs) for single trees, which also flags the root's x cut; a forest's
        // instance passes follow a full sort
        const bool full = t.sort_full || t.ninst > 1;
        uint8_t* side0 = !full && lglob > 0 ? t.d_sideX : nullptr;
        if ((st = sort_coordinates(t, s, xy, full, &src, side0, side0 ? t.seg_x[0].d_nzero : nullptr))) return st;
        marked = side0 != nullptr;
    } else {
        k_keys<<<nblk(n, 256), 256, 0, s>>>(xy, n, t.d_keys[0], t.d_keys[1], t.d_vals[0], t.d_vals[1], t.d_status);
        FMM_CUDA(cudaGetLastError());
        for (int pass = 0; pass < 8; ++pass) {
            if ((st = sort_pass(t, s, src, 2 - src, 8 * pass))) return st;
            src = 2 - src;
        }
    }
    if (t.ninst > 1) {
        k_inst_keys<<<nblk(n, 256), 256, 0, s>>>(t.d_vals[src], t.d_vals[src + 1], t.d_inst_ptoff, t.ninst, n,
                                                 t.d_keys[src], t.d_keys[src + 1]);
        for (int pass = 0; pass < 2; ++pass) {
            if ((st = sort_pass(t, s, src, 2 - src, 8 * pass))) return st;
            src = 2 - src;
        }
    }
    int32_t* X = t.d_vals[src];
    int32_t* Y = t.d_vals[src + 1];
    int32_t* X2 = t.d_X2;
    int32_t* Y2 = t.d_Y2;
    // geometry of level l from its lists: carried by the stage that cuts level l in x (which reads Y and
    // leaves X untouched); level lglob, which no global stage cuts, by k_geom
    auto geometry = [&](int l, const int32_t* Xl, const int32_t* Yl) {
        const LevelList& Ll = t.level_boxes[l];
        GeomArgs g;
        g.ids = Ll.d_ids;
        g.cnt = (int)Ll.count;
        g.X = Xl;
        g.Y = Yl;
        g.xy = xy;
        g.bstart = t.d_bstart;
        g.bcount = t.d_bcount;
        g.inst = t.d_inst;
        g.inst_box_off = t.d_inst_boxoff;
        g.center = t.d_center;
        g.radius = t.d_radius;
        g.rho = t.d_rho;
        g.chl = t.d_chl;
        g.rho32 = t.d_rho32;
        g.rad32 = t.d_rad32;
        g.is_root_level = l == 0 ? 1 : 0;
        return g;
    };
    GeomArgs none = geometry(0, X, Y);
    none.cnt = 0;
    if (lglob > 0 && !marked) {  // flags of the first cut (x, level 0); later cuts get theirs from the stage before
        const SegTable& sx = t.seg_x[0];
        launch_dep(true, k_mark, nblk(n, 256), 256, 0, s,
                   X, n, sx.d_start, sx.d_nzero, sx.K, t.d_sideX);
    }
    for (int l = 0; l < lglob; ++l) {
        const SegTable& sx = t.seg_x[l];
        const SegTable& sy = t.seg_y[l];
        // x-cut: Y partitioned by the x-side flags; the y-cut flags come from Y's new order
        if ((st = partition(t, s, 2 * l, Y, t.d_sideX, sx, Y2, &sy, t.d_sideY, geometry(l, X, Y)))) return st;
        std::swap(Y, Y2);
        // y-cut: X partitioned by the y-side flags; the next level's x-cut flags come from X's new order
        const SegTable* nxt = l + 1 < lglob ? &t.seg_x[l + 1] : nullptr;
        if ((st = partition(t, s, 2 * l + 1, X, t.d_sideY, sy, X2, nxt, t.d_sideX, none))) return st;
        std::swap(X, X2);
    }
    const GeomArgs gl = geometry(lglob, X, Y);
    if (gl.cnt > 0) {
        launch_dep(true, k_geom, nblk(gl.cnt, 128), 128, 0, s, gl);
        FMM_CUDA(cudaGetLastError());
    }
    if (lglob < t.Lmax - 1 && t.level_parents[lglob].count > 0) {
        // every remaining split inside one CTA per box of level l0
        const LevelList& Lp = t.level_parents[lglob];
        launch_dep(true, k_subtree, Lp.count, kSubThreads, 0, s,
                   Lp.d_ids, Lp.count, lglob, X, Y, xy, t.d_bstart, t.d_bcount, t.d_inst, t.d_inst_boxoff,
                   t.d_inst_levels, t.d_loc, t.d_center, t.d_radius, t.d_rho, t.d_chl, t.d_rho32, t.d_rad32,
                   t.d_status);
        FMM_CUDA(cudaGetLastError());
    }
    const bool f32 = t.path == FMM_PATH_FP32;
    if (t.n_src > 0)
        launch_dep(true, k_target_slots, nblk(32 * t.nleaf, 128), 128, 0, s,
                   t.leaves.d_ids, (int)t.nleaf, t.d_bstart, t.d_bcount, t.d_pslot, Y, (int)t.n_src, t.d_slot_of,
                   t.d_nsrc);
    launch_dep(true, k_finalize, nblk(n, 256), 256, 0, s,
               Y, n, xy, t.d_inst, t.d_inst_boxoff, t.d_center, t.d_perm, t.d_pts, t.d_pos4, t.d_leaf_of, t.d_slot_of,
               f32 ? static_cast<float*>(t.d_posp) : nullptr, f32 ? nullptr : static_cast<double2*>(t.d_posp));
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

fmm_status run_lists(Tree& t, cudaStream_t s) {
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(t.d_status) + 1;
    unsigned long long* need = t.d_lvl_base + 2 * kMaxLevels;
    FMM_CUDA(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), s));
    FMM_CUDA(cudaMemsetAsync(need, 0, 6 * sizeof(unsigned long long), s));
    const long long tiles_cap = t.cand_cap / kLTile + 2;
    const size_t lstride = (size_t)(2 * tiles_cap + 1);  // status words + ticket of one level
    FMM_CUDA(cudaMemsetAsync(t.d_ltstat, 0, lstride * (size_t)std::max(t.Lmax - 1, 1) * sizeof(unsigned long long),
                             s));
    FMM_CUDA(cudaMemsetAsync(t.d_m2l_rowctr, 0, (kM2LItemPairsMax + 4) * sizeof(unsigned long long), s));
    // P2P sources of a leaf: its points, or with separate evaluation points its sources only
    const int32_t* srccount = t.n_src > 0 ? t.d_nsrc : t.d_bcount;
    launch_dep(false, k_lists_root, nblk(t.ninst, 128), 128, 0, s,
               t.d_inst_boxoff, t.ninst, t.d_soff, t.d_ns, t.d_sidx, t.d_sowner, t.d_woff, t.d_nw, t.d_lvl_base,
               t.d_child0, t.d_pslot, srccount, t.d_srng);
    const int grid = t.num_sms * 8;
    for (int l = 1; l < t.Lmax; ++l) {
        launch_dep(true, k_lists_level, grid, kLThreads, 0, s,
                   l, t.d_lvl_base, t.d_sowner, t.d_soff, t.d_ns, t.d_sidx, t.d_woff, t.d_nw, t.d_widx, t.d_child0,
                   t.d_pslot, srccount, t.d_srng, t.d_chl, t.d_rad32, t.d_center, t.d_radius, t.theta,
                   t.d_ltstat + lstride * (size_t)(l - 1), tiles_cap, t.scap_tot, t.wcap_tot, need, t.d_status);
    }
    launch_dep(true, k_items, nblk(t.nbox, 128), 128, 0, s,
               (int)t.nbox, t.d_child0, t.d_bcount, t.d_soff, t.d_ns, t.d_woff, t.d_nw, ctr, t.d_p2p_items,
               t.d_p2p_rows, t.d_leaf_items, t.p2p_cap, t.d_m2l_items, t.d_box_m2l, t.m2l_cap, m2l_item_pairs(t),
               t.d_m2l_rowctr, t.d_m2l_rows, t.d_box_tail, t.d_status, p2p_item_sources(t.n));
    launch_dep(true, k_m2l_rows, nblk(t.nbox, 256), 256, 0, s,
               (int)t.nbox, t.d_box_m2l, t.d_box_tail, t.d_m2l_rowctr, t.m2l_cap, t.d_m2l_rows, ctr + 2, need,
               t.d_status);
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

fmm_status run_count(Tree& t, cudaStream_t s, unsigned long long out[2]) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(t.d_status) + 5;
    FMM_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s));
    k_count<<<nblk(t.nleaf, 256), 256, 0, s>>>(t.leaves.d_ids, (int)t.nleaf, t.d_soff, t.d_ns, t.d_sidx, t.d_bcount,
                                               cnt);
    FMM_CUDA(cudaGetLastError());
    FMM_CUDA(cudaMemcpyAsync(out, cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    return FMM_OK;
}

}  // namespace fmm
