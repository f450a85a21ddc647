// fmm_direct_eval_noalloc: the exact pairwise sum Phi(z_i) = sum_{z_j != z_i}
// Gamma_j/(z_i - z_j) for up to kNaMaxN points, computed by a variant of the
// library's P2P kernel (targets across lanes, sources split into chunks whose
// partial sums are added in a fixed order) WITHOUT allocating any device
// memory.
//
// Who needs this: code that runs inside a host application which owns every
// device allocation (a pre-sized pool handed out by a framework, a plug-in
// that must not grow the process's device footprint), and latency-critical
// loops where a cudaMalloc / cudaFree — which can synchronise the device and
// fragment such a pool — is not allowed.  These callers pass their own input
// and output buffers and get the result with no allocation on any path.
//
// The scratch for the partial sums is a file-scope __device__ array of fixed
// size (2 MiB), present on every GPU that loads the library until the process
// exits.  Every call shares it: calls whose kernels overlap on a GPU (for
// example on two streams without ordering between them) race on it and give
// wrong results; calls on one stream are safe.  Each call writes every scratch
// slot it later reads, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include "fmm_internal.cuh"

namespace {

constexpr int kNaMaxN = 16384;                 // largest accepted point count
constexpr int kNaTile = 32;                     // targets per warp item (one per lane)
constexpr int kNaChunk = 2048;                  // sources per warp item
constexpr int kNaTiles = kNaMaxN / kNaTile;     // 512
constexpr int kNaChunks = kNaMaxN / kNaChunk;   // 8
constexpr int kNaWarps = 8;

// partial sums: [tile][chunk][lane], complex128 -> 2 MiB
static __device__ __align__(256) double2 g_na_scratch[kNaTiles * kNaChunks * kNaTile];

// Device address of the scratch array on the current device.  In host code
// `g_na_scratch` names a host-side stand-in, never a device address, so kernels
// must be given the address cudaGetSymbolAddress returns.  It is looked up on
// every call (no allocation, no device synchronisation), so it stays right
// after a cudaDeviceReset reloads the module, and on every device.
fmm_status na_scratch(double2** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return fmm::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    *out = static_cast<double2*>(p);
    return FMM_OK;
}

// One warp per (target tile, source chunk): lane = target; the partial sum of
// the chunk goes to the scratch slot of (tile, chunk, lane).
__global__ void __launch_bounds__(kNaWarps * 32) k_na_partial(const double2* __restrict__ xy,
                                                              const double2* __restrict__ gam, int n, int nchunks,
                                                              double2* __restrict__ part) {
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int ntiles = (n + kNaTile - 1) / kNaTile;
    if (w >= ntiles * nchunks) return;
    const int tile = w / nchunks, chunk = w % nchunks;
    const int i = tile * kNaTile + lane;
    const double2 zt = i < n ? xy[i] : make_double2(0.0, 0.0);
    double2 acc = make_double2(0.0, 0.0);
    const int j1 = min(n, (chunk + 1) * kNaChunk);
    for (int j = chunk * kNaChunk; j < j1; ++j) {
        const double2 zs = xy[j];
        const double2 g = gam[j];
        const double dx = zt.x - zs.x, dy = zt.y - zs.y;
        const double r2 = fma(dx, dx, dy * dy);
        const double inv = r2 > 0.0 ? __drcp_rn(r2) : 0.0;  // z_j == z_i contributes nothing
        acc.x = fma(fma(g.x, dx, g.y * dy), inv, acc.x);
        acc.y = fma(fma(g.y, dx, -g.x * dy), inv, acc.y);
    }
    part[((size_t)tile * nchunks + chunk) * kNaTile + lane] = acc;
}

// Sum of the chunk partials of every target, in chunk order.
__global__ void k_na_reduce(int n, int nchunks, const double2* __restrict__ part, double2* __restrict__ phi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int tile = i / kNaTile, lane = i % kNaTile;
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) {
        const double2 v = part[((size_t)tile * nchunks + c) * kNaTile + lane];
        s.x += v.x;
        s.y += v.y;
    }
    phi[i] = s;
}

}  // namespace

extern "C" fmm_status fmm_direct_eval_noalloc(const double* d_xy, const double* d_gamma, int64_t n, double* d_phi,
                                              void* stream) {
    if (!d_xy || !d_gamma || !d_phi) {
        fmm::set_error("fmm_direct_eval_noalloc: NULL pointer");
        return FMM_ERR_INVALID_ARG;
    }
    if (n < 1 || n > kNaMaxN) {
        fmm::set_error("fmm_direct_eval_noalloc: n must be in [1, 16384] (fixed scratch size)");
        return FMM_ERR_INVALID_ARG;
    }
    double2* part = nullptr;
    fmm_status st = na_scratch(&part);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nn = (int)n;
    const int nchunks = (nn + kNaChunk - 1) / kNaChunk;
    const int items = ((nn + kNaTile - 1) / kNaTile) * nchunks;
    k_na_partial<<<(items + kNaWarps - 1) / kNaWarps, kNaWarps * 32, 0, s>>>(
        reinterpret_cast<const double2*>(d_xy), reinterpret_cast<const double2*>(d_gamma), nn, nchunks, part);
    k_na_reduce<<<(nn + 255) / 256, 256, 0, s>>>(nn, nchunks, part, reinterpret_cast<double2*>(d_phi));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fmm::cuda_fail(e, "fmm_direct_eval_noalloc launch");
    return FMM_OK;
}
