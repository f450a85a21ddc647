// FMM passes on the device (Sec. 2.1, Fig 2.2 of the paper): P2M, M2M, M2L,
// L2L, L2P and the P2P near-field sum for the harmonic kernel
//     Phi(z) = sum_j Gamma_j / (z - z_j).
//
// Expansions are stored SCALED by the box's scale radius rho, so that every
// ratio entering a shift is <= 1 in magnitude and FP32 never under/overflows:
//   multipole  M(z) = sum_k at_k rho^k / (z-c)^(k+1),  at_k = sum_j Gamma_j ((z_j-c)/rho)^k
//   local      L(z) = sum_l bt_l ((z-c)/rho)^l
// Shifts (all derived from the binomial series of the textbook expansions):
//   M2M  at'_n = sum_{k<=n} C(n,k) (sigma^k at_k) q^(n-k),   sigma = rho_c/rho_P, q = (c_c-c_P)/rho_P
//   M2L  bt_l += (-rho_L u)^l u sum_k C(k+l,l) (rho_M u)^k at_k,   u = 1/(c_L - c_M)
//   L2L  bt'_m = sigma^m sum_{l>=m} C(l,m) bt_l q^(l-m)
// M2M and L2L run as in-place Taylor shifts (p(p-1)/2 complex multiply-adds,
// no binomial table); M2L applies the binomial matrix with the coefficients
// C(k+l,l) folded into the instruction stream as immediates (p is a template
// parameter).
//
// Precision paths: FP32 path = P2M, M2L, L2P, P2P in FP32 (FP32 accumulation),
// M2M / L2L and the per-level local sums in FP64.  FP64 path = all FP64.
//
// Logarithmic kernel (Sec. 3.3), Phi(z) = sum_j q_j ln|z - z_j| for real q
// (complex strengths = two real-strength sets, one per part): with
// F(z) = sum_j q_j log(z - z_j), Re F = Phi and F' = the harmonic sum, so the
// log multipole q_0 log(z-c) + sum_k a_k/(z-c)^k is the integral of the
// harmonic one (a_k = -at_k rho^k / k) and the harmonic passes run unchanged
// on the same coefficients.  Only the constant term of each local expansion is
// new (slot P of the coefficient stride, real part only: the imaginary part of
// log is branch-dependent and never reaches Re F):
//   M2L  b0 += Re(at_0) ln|c_L - c_M| - sum_{k>=1} Re(v_k) / k,   v_k = (rho_M u)^k at_k
//   L2L  b0' = b0 + rho_P Re( q sum_m bt_m q^m / (m+1) )           (parent's polynomial at c_child)
//   L2P  F   = b0 + rho   Re( w sum_m bt_m w^m / (m+1) )
// which is the textbook log-series FMM with locals of degree p, exactly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

static inline int nblk(int64_t n, int b) { return (int)std::max<int64_t>((n + b - 1) / b, 1); }

// Binomial coefficients C(n,k), n < 64, k < 32, by Pascal's rule at compile
// time; kernels index them with unrolled (compile-time) indices.
struct BinomTable {
    float f[64][32];
    double d[64][32];
};
static constexpr BinomTable make_binom() {
    BinomTable t{};
    double row[64] = {};
    for (int n = 0; n < 64; ++n) {
        for (int k = n; k >= 1; --k) row[k] = row[k] + row[k - 1];
        row[0] = 1.0;
        for (int k = 0; k < 32; ++k) {
            t.d[n][k] = k <= n ? row[k] : 0.0;
            t.f[n][k] = (float)t.d[n][k];
        }
    }
    return t;
}
__constant__ BinomTable c_binom = make_binom();

// n! and 1/n! for n < 32 (lane-indexed by the warp-per-shift kernels).
struct FactTable {
    double f[32];
    double inv[32];
};
static constexpr FactTable make_fact() {
    FactTable t{};
    double x = 1.0;
    for (int n = 0; n < 32; ++n) {
        if (n > 0) x *= n;
        t.f[n] = x;
        t.inv[n] = 1.0 / x;
    }
    return t;
}
__constant__ FactTable c_fact = make_fact();

// ------------------------------------------------------------------ gather

// Strengths into sorted order and into the leaf slot layout of the P2P pass
// (FP32: slot pairs interleaved as (re[2m], re[2m+1], im[2m], im[2m+1])).
__device__ __forceinline__ void d_gather32(const int vbx, const double2* __restrict__ in, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ slot_of, int n, float2* out, float* outp, unsigned* cplx) {
    const int i = vbx * blockDim.x + threadIdx.x;
    bool im = false;
    if (i < n) {
        const double2 g = in[perm[i]];
        const float2 v = make_float2((float)g.x, (float)g.y);
        out[i] = v;
        const int slot = slot_of[i];
        float* f = outp + 4 * (slot >> 1) + (slot & 1);
        f[0] = v.x;
        f[2] = v.y;
        im = v.y != 0.f;
    }
    // record complex strengths: one plain store per block that saw one (every writer stores the same value)
    if (cplx != nullptr && __syncthreads_or(im) && threadIdx.x == 0) *cplx = 1u;
}
__global__ void k_gather32(const double2* __restrict__ in, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ slot_of, int n, float2* out, float* outp, unsigned* cplx) { d_gather32(blockIdx.x, in, perm, slot_of, n, out, outp, cplx); }
__global__ void k_gather64(const double2* __restrict__ in, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ slot_of, int n, double2* out, double2* outp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 g = in[perm[i]];
    out[i] = g;
    outp[slot_of[i]] = g;
}

// Logarithmic kernel: the real and imaginary parts of the strengths become two
// real-strength sets for the far field (sorted order, imaginary part zero);
// the P2P slot layout keeps the complex strengths (one log per pair).
__global__ void k_gather_log32(const double2* __restrict__ in, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ slot_of, int n, float2* out0, float2* out1,
                               float* outp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 g = in[perm[i]];
    const float2 v = make_float2((float)g.x, (float)g.y);
    out0[i] = make_float2(v.x, 0.f);
    out1[i] = make_float2(v.y, 0.f);
    const int slot = slot_of[i];
    float* f = outp + 4 * (slot >> 1) + (slot & 1);
    f[0] = v.x;
    f[2] = v.y;
}
__global__ void k_gather_log64(const double2* __restrict__ in, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ slot_of, int n, double2* out0, double2* out1,
                               double2* outp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 g = in[perm[i]];
    out0[i] = make_double2(g.x, 0.0);
    out1[i] = make_double2(g.y, 0.0);
    outp[slot_of[i]] = g;
}

// --------------------------------------------------------------------- P2M

// One thread per leaf: at_k = sum_j Gamma_j w_j^k, w_j = (z_j - c)/rho, FP32.
// Point offsets use the hi/lo split so w keeps full FP32 accuracy.
template <int P>
__device__ __forceinline__ void d_p2m32(const int vbx, const int32_t* __restrict__ leaves, int nleaf,
                                               const int32_t* __restrict__ bstart, const int32_t* __restrict__ bcount,
                                               const float4* __restrict__ chl, const float* __restrict__ rho32,
                                               const float4* __restrict__ pos4, const float2* __restrict__ gam,
                                               float2* __restrict__ M32, double2* __restrict__ M64, int p, int PS) {
    int q = vbx * blockDim.x + threadIdx.x;
    if (q >= nleaf) return;
    const int b = leaves[q];
    const float4 c = chl[b];
    const float r = rho32[b];
    const float inv = r > 0.f ? 1.0f / r : 0.f;
    float2 a[P];
#pragma unroll
    for (int k = 0; k < P; ++k) a[k] = make_float2(0.f, 0.f);
    const int s = bstart[b], e = s + bcount[b];
    for (int i = s; i < e; ++i) {
        const float4 pt = pos4[i];
        const float2 w = make_float2(((pt.x - c.x) + (pt.z - c.z)) * inv, ((pt.y - c.y) + (pt.w - c.w)) * inv);
        float2 t = gam[i];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            a[k].x += t.x;
            a[k].y += t.y;
            t = cmul(t, w);
        }
    }
    float2* out = M32 + (size_t)b * PS;
#pragma unroll
    for (int k = 0; k < P; ++k) out[k] = k < p ? a[k] : make_float2(0.f, 0.f);
    if (M64 != nullptr) {  // a parent box: the FP64 copy that the next shift up reads
        double2* o64 = M64 + (size_t)b * PS;
#pragma unroll
        for (int k = 0; k < P; ++k) o64[k] = k < p ? make_double2((double)a[k].x, (double)a[k].y) : make_double2(0.0, 0.0);
    }
}
template <int P>
__global__ void __launch_bounds__(128) k_p2m32(const int32_t* __restrict__ leaves, int nleaf,
                                               const int32_t* __restrict__ bstart, const int32_t* __restrict__ bcount,
                                               const float4* __restrict__ chl, const float* __restrict__ rho32,
                                               const float4* __restrict__ pos4, const float2* __restrict__ gam,
                                               float2* __restrict__ M32, double2* __restrict__ M64, int p, int PS) { d_p2m32<P>(blockIdx.x, leaves, nleaf, bstart, bcount, chl, rho32, pos4, gam, M32, M64, p, PS); }

// P2M of boxes with up to ~1024 points: one warp per box, lanes over its points,
// then an xor-butterfly over the lanes (a fixed order); writes the FP32
// multipole and its FP64 copy (these boxes are parents, read by the next shift).
template <int P>
__device__ __forceinline__ void d_p2m32_warp(const int vbx, const int32_t* __restrict__ boxes, int cnt,
                                                    const int32_t* __restrict__ bstart,
                                                    const int32_t* __restrict__ bcount, const float4* __restrict__ chl,
                                                    const float* __restrict__ rho32, const float4* __restrict__ pos4,
                                                    const float2* __restrict__ gam, float2* __restrict__ M32,
                                                    double2* __restrict__ M64, int p, int PS) {
    const int w = (int)((vbx * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= cnt) return;  // warp-uniform
    const int b = boxes[w];
    const float4 c = chl[b];
    const float r = rho32[b];
    const float inv = r > 0.f ? 1.0f / r : 0.f;
    float2 a[P];
#pragma unroll
    for (int k = 0; k < P; ++k) a[k] = make_float2(0.f, 0.f);
    const int s = bstart[b], e = s + bcount[b];
    for (int i = s + lane; i < e; i += 32) {
        const float4 pt = pos4[i];
        const float2 wv = make_float2(((pt.x - c.x) + (pt.z - c.z)) * inv, ((pt.y - c.y) + (pt.w - c.w)) * inv);
        float2 t = gam[i];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            a[k].x += t.x;
            a[k].y += t.y;
            t = cmul(t, wv);
        }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a[k].x += __shfl_xor_sync(0xffffffffu, a[k].x, o);
            a[k].y += __shfl_xor_sync(0xffffffffu, a[k].y, o);
        }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (lane == (k & 31)) {
            const float2 v = k < p ? a[k] : make_float2(0.f, 0.f);
            M32[(size_t)b * PS + k] = v;
            M64[(size_t)b * PS + k] = make_double2((double)v.x, (double)v.y);
        }
    }
}
template <int P>
__global__ void __launch_bounds__(128) k_p2m32_warp(const int32_t* __restrict__ boxes, int cnt,
                                                    const int32_t* __restrict__ bstart,
                                                    const int32_t* __restrict__ bcount, const float4* __restrict__ chl,
                                                    const float* __restrict__ rho32, const float4* __restrict__ pos4,
                                                    const float2* __restrict__ gam, float2* __restrict__ M32,
                                                    double2* __restrict__ M64, int p, int PS) { d_p2m32_warp<P>(blockIdx.x, boxes, cnt, bstart, bcount, chl, rho32, pos4, gam, M32, M64, p, PS); }

template <int P>
__global__ void __launch_bounds__(128) k_p2m64(const int32_t* __restrict__ leaves, int nleaf,
                                               const int32_t* __restrict__ bstart, const int32_t* __restrict__ bcount,
                                               const double2* __restrict__ center, const double* __restrict__ rho,
                                               const double2* __restrict__ pts, const double2* __restrict__ gam,
                                               double2* __restrict__ M64, int p, int PS) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nleaf) return;
    const int b = leaves[q];
    const double2 c = center[b];
    const double r = rho[b];
    const double inv = r > 0.0 ? 1.0 / r : 0.0;
    double2 a[P];
#pragma unroll
    for (int k = 0; k < P; ++k) a[k] = make_double2(0.0, 0.0);
    const int s = bstart[b], e = s + bcount[b];
    for (int i = s; i < e; ++i) {
        const double2 pt = pts[i];
        const double2 w = make_double2((pt.x - c.x) * inv, (pt.y - c.y) * inv);
        double2 t = gam[i];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            a[k].x += t.x;
            a[k].y += t.y;
            t = cmul(t, w);
        }
    }
    double2* out = M64 + (size_t)b * PS;
#pragma unroll
    for (int k = 0; k < P; ++k) out[k] = k < p ? a[k] : make_double2(0.0, 0.0);
}

// --------------------------------------------------------------------- M2M

// One thread per (parent, child), FP64: four consecutive lanes shift the four
// children of one parent and add them with two xor-shuffles (fixed order).
// Leaf children of the FP32 path are read from the FP32 multipoles of P2M.
template <int P>
__device__ __forceinline__ void d_m2m(const int vbx, const int32_t* __restrict__ parents, int cnt,
                                             const int32_t* __restrict__ child0, const double* __restrict__ rho,
                                             const double2* __restrict__ center, const float2* __restrict__ M32in,
                                             double2* __restrict__ M64, float2* __restrict__ M32out, int fp32_path,
                                             int p, int PS) {
    const int q = vbx * blockDim.x + threadIdx.x;
    const int pi = q >> 2, c = q & 3;
    const bool valid = pi < cnt;
    double2 v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = make_double2(0.0, 0.0);
    int b = 0;
    if (valid) {
        b = parents[pi];
        const int h = child0[b] + c;
        const double rP = rho[b];
        const double inv = rP > 0.0 ? 1.0 / rP : 0.0;
        if (fp32_path && child0[h] < 0) {
            const float2* src = M32in + (size_t)h * PS;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float2 f = src[k];
                v[k] = make_double2((double)f.x, (double)f.y);
            }
        } else {
            const double2* src = M64 + (size_t)h * PS;
#pragma unroll
            for (int k = 0; k < P; ++k) v[k] = src[k];
        }
        const double sigma = rho[h] * inv;
        const double2 cP = center[b], ch = center[h];
        const double2 qv = make_double2((ch.x - cP.x) * inv, (ch.y - cP.y) * inv);
        double sp = 1.0;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            v[k].x *= sp;
            v[k].y *= sp;
            sp *= sigma;
        }
        // in-place Taylor shift: after the sweeps v_n = sum_{k<=n} C(n,k) v_k q^(n-k)
#pragma unroll
        for (int k = P - 1; k >= 1; --k) {
#pragma unroll
            for (int j = k; j < P; ++j) v[j] = cfma(qv, v[j - 1], v[j]);
        }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
        v[k].x += __shfl_xor_sync(0xffffffffu, v[k].x, 1);
        v[k].y += __shfl_xor_sync(0xffffffffu, v[k].y, 1);
        v[k].x += __shfl_xor_sync(0xffffffffu, v[k].x, 2);
        v[k].y += __shfl_xor_sync(0xffffffffu, v[k].y, 2);
    }
    if (!valid || c != 0) return;
    // the shift fills orders >= p from lower ones: keep the expansion at p terms
    double2* out = M64 + (size_t)b * PS;
#pragma unroll
    for (int k = 0; k < P; ++k) out[k] = k < p ? v[k] : make_double2(0.0, 0.0);
    if (fp32_path) {
        float2* o32 = M32out + (size_t)b * PS;
#pragma unroll
        for (int k = 0; k < P; ++k) o32[k] = k < p ? make_float2((float)v[k].x, (float)v[k].y) : make_float2(0.f, 0.f);
    }
}
template <int P>
__global__ void __launch_bounds__(128) k_m2m(const int32_t* __restrict__ parents, int cnt,
                                             const int32_t* __restrict__ child0, const double* __restrict__ rho,
                                             const double2* __restrict__ center, const float2* __restrict__ M32in,
                                             double2* __restrict__ M64, float2* __restrict__ M32out, int fp32_path,
                                             int p, int PS) { d_m2m<P>(blockIdx.x, parents, cnt, child0, rho, center, M32in, M64, M32out, fp32_path, p, PS); }

// --------------------------------------------------------------------- M2L

// One thread per target box (every level in one launch), looping over the
// box's weak list.  FP32 with FP32 accumulation.  Root boxes (no parent) also
// seed the FP64 local array, which L2L reads for level 1.
// Binomial coefficients as compile-time constants: the unrolled M2L applies
// C(k+l, l) as FFMA immediates (no constant-bank loads in the inner loop).
template <int N, int K>
struct Bn {
    static constexpr float v = (float)binom_d(N, K);
};

template <int P, int K, int... L>
__device__ __forceinline__ void m2l_row(float2 (&w)[P], const float2 v, std::integer_sequence<int, L...>) {
    ((w[L].x = fmaf(Bn<K + L, L>::v, v.x, w[L].x)), ...);
    ((w[L].y = fmaf(Bn<K + L, L>::v, v.y, w[L].y)), ...);
}

template <int P, int K, bool LOG>
__device__ __forceinline__ void m2l_step(float2 (&w)[P], const float4 (&aa)[(P + 1) / 2], float2& ap,
                                         const float2 alpha, float& ls) {
    const float4 q = aa[K / 2];
    const float2 a = (K & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
    const float2 v = cmul(ap, a);
    if (K + 1 < P) ap = cmul(ap, alpha);
    if constexpr (LOG && K >= 1) ls = fmaf(-1.0f / K, v.x, ls);  // log kernel: -sum_k Re(v_k)/k
    m2l_row<P, K>(w, v, std::make_integer_sequence<int, P>{});
}

// w_l = sum_k C(k+l, l) alpha^k a_k for l < P (a_k held in registers)
template <int P, bool LOG, int... K>
__device__ __forceinline__ void m2l_apply(float2 (&w)[P], const float4 (&aa)[(P + 1) / 2], const float2 alpha,
                                          float& ls, std::integer_sequence<int, K...>) {
    float2 ap = make_float2(1.f, 0.f);
    (m2l_step<P, K, LOG>(w, aa, ap, alpha, ls), ...);
}

template <int P, bool LOG>
__device__ __forceinline__ void d_m2l32(const int vbx, const int4* __restrict__ items,
                                               const unsigned long long* __restrict__ nitems,
                                               const int32_t* __restrict__ woff, const int32_t* __restrict__ widx,
                                               const float4* __restrict__ chl, const float* __restrict__ rho32,
                                               const float2* __restrict__ M32, float2* __restrict__ Lm2l,
                                               float2* __restrict__ part, const int32_t* __restrict__ rows, int PS) {
    const int row = vbx * blockDim.x + threadIdx.x;
    if (row >= (int)*nitems) return;
    const int it = rows[row];  // work item of this thread (row order: similar lengths within a warp)
    const int4 item = items[it];
    const int b = item.x;
    const float4 ct = chl[b];
    const float rt = rho32[b];
    float2 acc[P];
#pragma unroll
    for (int l = 0; l < P; ++l) acc[l] = make_float2(0.f, 0.f);
    float b0 = 0.f;  // log kernel: constant term
    const int32_t* wl = widx + woff[b];
    for (int j = item.y; j < item.z; ++j) {
        const int s = wl[j];
        const float4 cs = chl[s];
        const float rs = rho32[s];
        const float dx = (ct.x - cs.x) + (ct.z - cs.z);
        const float dy = (ct.y - cs.y) + (ct.w - cs.w);
        const float r2 = fmaf(dx, dx, dy * dy);
        const float inv = 1.0f / r2;
        const float2 u = make_float2(dx * inv, -dy * inv);  // 1/d, d = c_target - c_source
        const float2 alpha = make_float2(rs * u.x, rs * u.y);
        const float2 beta = make_float2(-rt * u.x, -rt * u.y);
        float2 w[P];
#pragma unroll
        for (int l = 0; l < P; ++l) w[l] = make_float2(0.f, 0.f);
        float4 aa[(P + 1) / 2];
        const float4* src = reinterpret_cast<const float4*>(M32 + (size_t)s * PS);
#pragma unroll
        for (int k2 = 0; k2 < (P + 1) / 2; ++k2) aa[k2] = src[k2];
        float ls = 0.f;
        m2l_apply<P, LOG>(w, aa, alpha, ls, std::make_integer_sequence<int, P>{});
        if constexpr (LOG) b0 += fmaf(0.5f * logf(r2), aa[0].x, ls);
        float2 g = u;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            acc[l] = cfma(g, w[l], acc[l]);
            g = cmul(g, beta);
        }
    }
    float2* out = item.w < 0 ? Lm2l + (size_t)b * PS : part + (size_t)it * PS;
#pragma unroll
    for (int l = 0; l < P; ++l) out[l] = acc[l];
    if constexpr (LOG) out[P] = make_float2(b0, 0.f);
}
template <int P, bool LOG>
__global__ void __launch_bounds__(128) k_m2l32(const int4* __restrict__ items,
                                               const unsigned long long* __restrict__ nitems,
                                               const int32_t* __restrict__ woff, const int32_t* __restrict__ widx,
                                               const float4* __restrict__ chl, const float* __restrict__ rho32,
                                               const float2* __restrict__ M32, float2* __restrict__ Lm2l,
                                               float2* __restrict__ part, const int32_t* __restrict__ rows, int PS) { d_m2l32<P, LOG>(blockIdx.x, items, nitems, woff, widx, chl, rho32, M32, Lm2l, part, rows, PS); }

template <int P, bool LOG>
__global__ void __launch_bounds__(128) k_m2l64(const int4* __restrict__ items,
                                               const unsigned long long* __restrict__ nitems,
                                               const int32_t* __restrict__ woff, const int32_t* __restrict__ widx,
                                               const double2* __restrict__ center, const double* __restrict__ rho,
                                               const double2* __restrict__ M64, double2* __restrict__ Lm2l,
                                               double2* __restrict__ part, const int32_t* __restrict__ rows, int PS) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (int)*nitems) return;
    const int it = rows[row];  // work item of this thread (row order: similar lengths within a warp)
    const int4 item = items[it];
    const int b = item.x;
    const double2 ct = center[b];
    const double rt = rho[b];
    double2 acc[P];
#pragma unroll
    for (int l = 0; l < P; ++l) acc[l] = make_double2(0.0, 0.0);
    double b0 = 0.0;  // log kernel: constant term
    const int32_t* wl = widx + woff[b];
    for (int j = item.y; j < item.z; ++j) {
        const int s = wl[j];
        const double2 cs = center[s];
        const double rs = rho[s];
        const double dx = ct.x - cs.x, dy = ct.y - cs.y;
        const double r2 = dx * dx + dy * dy;
        const double inv = 1.0 / r2;
        const double2 u = make_double2(dx * inv, -dy * inv);
        const double2 alpha = make_double2(rs * u.x, rs * u.y);
        const double2 beta = make_double2(-rt * u.x, -rt * u.y);
        double2 w[P];
#pragma unroll
        for (int l = 0; l < P; ++l) w[l] = make_double2(0.0, 0.0);
        const double2* src = M64 + (size_t)s * PS;
        double2 ap = make_double2(1.0, 0.0);
        double ls = 0.0;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const double2 v = cmul(ap, src[k]);
            ap = cmul(ap, alpha);
            if (LOG && k >= 1) ls = fma(-1.0 / k, v.x, ls);
#pragma unroll
            for (int l = 0; l < P; ++l) {
                const double cb = c_binom.d[k + l][l];
                w[l].x = fma(cb, v.x, w[l].x);
                w[l].y = fma(cb, v.y, w[l].y);
            }
        }
        if constexpr (LOG) b0 += fma(0.5 * log(r2), src[0].x, ls);
        double2 g = u;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            acc[l] = cfma(g, w[l], acc[l]);
            g = cmul(g, beta);
        }
    }
    double2* out = item.w < 0 ? Lm2l + (size_t)b * PS : part + (size_t)it * PS;
#pragma unroll
    for (int l = 0; l < P; ++l) out[l] = acc[l];
    if constexpr (LOG) out[P] = make_double2(b0, 0.0);
}

// --------------------------------------------------------------------- L2L

// One thread per child box of one level; FP64.  child = shift(parent) + its
// own M2L sum.  In the FP32 path leaves also get an FP32 copy for L2P.  With
// LOG the constant term (slot P) is the parent's log polynomial at the child
// centre plus the child's own M2L constant.
template <int P, typename LM, bool LOG>
__device__ __forceinline__ void d_l2l(const int vbx, const int32_t* __restrict__ boxes, int cnt,
                                             const int32_t* __restrict__ parent, const int32_t* __restrict__ child0,
                                             const double* __restrict__ rho, const double2* __restrict__ center,
                                             const int2* __restrict__ box_m2l, const LM* __restrict__ Lm2l,
                                             double2* __restrict__ L64,
                                             float2* __restrict__ L32, int all32, int p, int PS) {
    int qi = vbx * blockDim.x + threadIdx.x;
    if (qi >= cnt) return;
    const int c = boxes[qi];
    const int Pb = parent[c];
    const double rP = rho[Pb];
    const double inv = rP > 0.0 ? 1.0 / rP : 0.0;
    const double2 cP = center[Pb], cc = center[c];
    const double2 q = make_double2((cc.x - cP.x) * inv, (cc.y - cP.y) * inv);
    const double sigma = rho[c] * inv;
    double2 b[P];
    const double2* src = L64 + (size_t)Pb * PS;
#pragma unroll
    for (int k = 0; k < P; ++k) b[k] = src[k];
    const int2 mi = box_m2l[c];
    const LM* o = Lm2l + (size_t)c * PS;
    double b0 = 0.0;
    if constexpr (LOG) {
        // Horner: h = sum_m bt_m q^m / (m+1); b0' = b0 + rho_P Re(q h) + own
        double2 h = make_double2(b[P - 1].x * (1.0 / P), b[P - 1].y * (1.0 / P));
#pragma unroll
        for (int m = P - 2; m >= 0; --m)
            h = cfma(h, q, make_double2(b[m].x * (1.0 / (m + 1)), b[m].y * (1.0 / (m + 1))));
        b0 = fma(rP, q.x * h.x - q.y * h.y, src[P].x);
        if (mi.y > 0) b0 += (double)o[P].x;
    }
    // in-place Taylor shift: after the sweeps b_m = sum_{l>=m} C(l,m) b_l q^(l-m)
#pragma unroll
    for (int k = 0; k + 1 < P; ++k) {
#pragma unroll
        for (int j = P - 2; j >= k; --j) b[j] = cfma(q, b[j + 1], b[j]);
    }
    // this box's own M2L sum (split boxes were summed by k_reduce_m2l)
    double2 own[P];
#pragma unroll
    for (int m = 0; m < P; ++m) own[m] = mi.y > 0 ? make_double2((double)o[m].x, (double)o[m].y) : make_double2(0.0, 0.0);
    double sp = 1.0;
    double2* out = L64 + (size_t)c * PS;
    const bool leaf32 = (L32 != nullptr) && (all32 || child0[c] < 0);
    float2* o32 = L32 + (size_t)c * PS;
#pragma unroll
    for (int m = 0; m < P; ++m) {
        double2 v = make_double2(fma(b[m].x, sp, own[m].x), fma(b[m].y, sp, own[m].y));
        if (m >= p) v = make_double2(0.0, 0.0);
        sp *= sigma;
        out[m] = v;
        if (leaf32) o32[m] = make_float2((float)v.x, (float)v.y);
    }
    if constexpr (LOG) {
        out[P] = make_double2(b0, 0.0);
        if (leaf32) o32[P] = make_float2((float)b0, 0.f);
    }
}
template <int P, typename LM, bool LOG>
__global__ void __launch_bounds__(128) k_l2l(const int32_t* __restrict__ boxes, int cnt,
                                             const int32_t* __restrict__ parent, const int32_t* __restrict__ child0,
                                             const double* __restrict__ rho, const double2* __restrict__ center,
                                             const int2* __restrict__ box_m2l, const LM* __restrict__ Lm2l,
                                             double2* __restrict__ L64,
                                             float2* __restrict__ L32, int all32, int p, int PS) { d_l2l<P, LM, LOG>(blockIdx.x, boxes, cnt, parent, child0, rho, center, box_m2l, Lm2l, L64, L32, all32, p, PS); }

// ---- M2M / L2L for levels with few boxes: one warp per shift -----------------
// FP64 warp instructions are expensive per issue on this GPU (the FP64 pipe
// takes many cycles per warp instruction whatever the number of active
// lanes), so a level with few boxes run as one thread per shift is bound by
// one warp's ~p^2/2 complex FMAs.  Here lane n computes output coefficient n
// of one shift as a convolution,
//   M2M  at'_n = n! sum_{k<=n} (sigma^k at_k / k!) (q^(n-k) / (n-k)!)
//   L2L  bt'_m = (sigma^m / m!) sum_{l>=m} (l! bt_l) (q^(l-m) / (l-m)!)
// (the binomial shifts of the header comment with C(n,k) = n!/(k!(n-k)!)),
// with the powers of sigma and q from a scan across lanes: ~p complex FMAs
// per lane spread over many warps.

// a_lane = x^lane by a Hillis-Steele product scan across the warp
__device__ __forceinline__ double2 lane_pow(double2 x, int lane) {
    double2 a = lane == 0 ? make_double2(1.0, 0.0) : x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double2 y = make_double2(__shfl_up_sync(0xffffffffu, a.x, d), __shfl_up_sync(0xffffffffu, a.y, d));
        if (lane >= d) a = cmul(a, y);
    }
    return a;
}
__device__ __forceinline__ double lane_pow(double x, int lane) {
    double a = lane == 0 ? 1.0 : x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, a, d);
        if (lane >= d) a *= y;
    }
    return a;
}
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// One CTA of 4 warps per parent; warp c shifts child c, and the four shifted
// expansions are added in a fixed order ((c0 + c1) + (c2 + c3)).
template <int P>
__device__ __forceinline__ void d_m2m_warp(const int vbx, const int32_t* __restrict__ parents, int cnt,
                                                  const int32_t* __restrict__ child0, const double* __restrict__ rho,
                                                  const double2* __restrict__ center,
                                                  const float2* __restrict__ M32in, double2* __restrict__ M64,
                                                  float2* __restrict__ M32out, int fp32_path, int p, int PS) {
    __shared__ double2 part[4][32];
    const int pi = vbx;
    if (pi >= cnt) return;
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = parents[pi];
    const int h = child0[b] + c;
    const double rP = rho[b];
    const double inv = rP > 0.0 ? 1.0 / rP : 0.0;
    const double sigma = rho[h] * inv;
    const double2 cP = center[b], ch = center[h];
    const double2 q = make_double2((ch.x - cP.x) * inv, (ch.y - cP.y) * inv);
    double2 v = make_double2(0.0, 0.0);
    if (lane < P) {
        if (fp32_path && child0[h] < 0) {
            const float2 f = M32in[(size_t)h * PS + lane];
            v = make_double2((double)f.x, (double)f.y);
        } else {
            v = M64[(size_t)h * PS + lane];
        }
    }
    const double sk = lane_pow(sigma, lane);
    const double2 qk = lane_pow(q, lane);
    const double ifk = c_fact.inv[lane];
    const double ys = sk * ifk;
    const double2 y = make_double2(v.x * ys, v.y * ys);
    const double2 z = make_double2(qk.x * ifk, qk.y * ifk);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const double2 yk = shfl2(y, k);
        const double2 zz = shfl2(z, (lane - k) & 31);
        if (k <= lane) acc = cfma(yk, zz, acc);
    }
    const double fn = c_fact.f[lane];
    part[c][lane] = make_double2(acc.x * fn, acc.y * fn);
    __syncthreads();
    if (c != 0 || lane >= P) return;
    const double2 s01 = make_double2(part[0][lane].x + part[1][lane].x, part[0][lane].y + part[1][lane].y);
    const double2 s23 = make_double2(part[2][lane].x + part[3][lane].x, part[2][lane].y + part[3][lane].y);
    const double2 s = lane < p ? make_double2(s01.x + s23.x, s01.y + s23.y) : make_double2(0.0, 0.0);
    M64[(size_t)b * PS + lane] = s;
    if (fp32_path) M32out[(size_t)b * PS + lane] = make_float2((float)s.x, (float)s.y);
}
template <int P>
__global__ void __launch_bounds__(128) k_m2m_warp(const int32_t* __restrict__ parents, int cnt,
                                                  const int32_t* __restrict__ child0, const double* __restrict__ rho,
                                                  const double2* __restrict__ center,
                                                  const float2* __restrict__ M32in, double2* __restrict__ M64,
                                                  float2* __restrict__ M32out, int fp32_path, int p, int PS) { d_m2m_warp<P>(blockIdx.x, parents, cnt, child0, rho, center, M32in, M64, M32out, fp32_path, p, PS); }

// One warp per child box: shifted parent local + the box's own M2L sum.  With
// LOG, lane m adds bt_m q^(m+1)/(m+1) to the constant term (xor-butterfly sum
// across the warp, a fixed order).
template <int P, typename LM, bool LOG>
__device__ __forceinline__ void d_l2l_warp(const int vbx, const int32_t* __restrict__ boxes, int cnt,
                                                  const int32_t* __restrict__ parent,
                                                  const int32_t* __restrict__ child0, const double* __restrict__ rho,
                                                  const double2* __restrict__ center,
                                                  const int2* __restrict__ box_m2l, const LM* __restrict__ Lm2l,
                                                  double2* __restrict__ L64, float2* __restrict__ L32, int all32, int p,
                                                  int PS) {
    const int qi = (int)((vbx * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (qi >= cnt) return;  // warp-uniform
    const int c = boxes[qi];
    const int Pb = parent[c];
    const double rP = rho[Pb];
    const double inv = rP > 0.0 ? 1.0 / rP : 0.0;
    const double2 cP = center[Pb], cc = center[c];
    const double2 q = make_double2((cc.x - cP.x) * inv, (cc.y - cP.y) * inv);
    const double sigma = rho[c] * inv;
    const double2 bl = lane < P ? L64[(size_t)Pb * PS + lane] : make_double2(0.0, 0.0);
    const double sk = lane_pow(sigma, lane);
    const double2 qk = lane_pow(q, lane);
    const double fl = c_fact.f[lane], ifl = c_fact.inv[lane];
    const double2 y = make_double2(bl.x * fl, bl.y * fl);
    const double2 z = make_double2(qk.x * ifl, qk.y * ifl);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int l = 0; l < P; ++l) {
        const double2 yl = shfl2(y, l);
        const double2 zz = shfl2(z, (l - lane) & 31);
        if (l >= lane) acc = cfma(yl, zz, acc);
    }
    const int2 mi = box_m2l[c];
    if constexpr (LOG) {
        const double2 q1 = cmul(qk, q);  // q^(lane+1)
        double t = (bl.x * q1.x - bl.y * q1.y) / (double)(lane + 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            double b0 = fma(rP, t, L64[(size_t)Pb * PS + P].x);
            if (mi.y > 0) b0 += (double)Lm2l[(size_t)c * PS + P].x;
            L64[(size_t)c * PS + P] = make_double2(b0, 0.0);
            if (L32 != nullptr && (all32 || child0[c] < 0)) L32[(size_t)c * PS + P] = make_float2((float)b0, 0.f);
        }
    }
    if (lane >= P) return;
    const double scale = sk * ifl;
    double2 own = make_double2(0.0, 0.0);
    if (mi.y > 0) {
        const LM o = Lm2l[(size_t)c * PS + lane];
        own = make_double2((double)o.x, (double)o.y);
    }
    double2 v = make_double2(fma(acc.x, scale, own.x), fma(acc.y, scale, own.y));
    if (lane >= p) v = make_double2(0.0, 0.0);
    L64[(size_t)c * PS + lane] = v;
    if (L32 != nullptr && (all32 || child0[c] < 0)) L32[(size_t)c * PS + lane] = make_float2((float)v.x, (float)v.y);
}
template <int P, typename LM, bool LOG>
__global__ void __launch_bounds__(128) k_l2l_warp(const int32_t* __restrict__ boxes, int cnt,
                                                  const int32_t* __restrict__ parent,
                                                  const int32_t* __restrict__ child0, const double* __restrict__ rho,
                                                  const double2* __restrict__ center,
                                                  const int2* __restrict__ box_m2l, const LM* __restrict__ Lm2l,
                                                  double2* __restrict__ L64, float2* __restrict__ L32, int all32, int p,
                                                  int PS) { d_l2l_warp<P, LM, LOG>(blockIdx.x, boxes, cnt, parent, child0, rho, center, box_m2l, Lm2l, L64, L32, all32, p, PS); }

// FP64 M2L with one warp per work item, for trees with few items (one thread
// per item would leave most of the GPU idle: a 1e4-point tree has ~340 items):
// lane l < P owns output coefficient l.  Per pair, lane k forms v_k = alpha^k
// at_k (the powers by a product scan across the lanes), w_l = sum_k C(k+l, l)
// v_k takes v_k from lane k by shuffles (k ascending, as in k_m2l64), and
// g_l = u beta^l scales it into the lane's sum.
template <int P, bool LOG>
__global__ void __launch_bounds__(128) k_m2l64_warp(const int4* __restrict__ items,
                                                    const unsigned long long* __restrict__ nitems,
                                                    const int32_t* __restrict__ woff,
                                                    const int32_t* __restrict__ widx,
                                                    const double2* __restrict__ center,
                                                    const double* __restrict__ rho, const double2* __restrict__ M64,
                                                    double2* __restrict__ Lm2l, double2* __restrict__ part,
                                                    const int32_t* __restrict__ rows, int PS) {
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= (int)*nitems) return;  // warp-uniform
    const int it = rows[row];
    const int4 item = items[it];
    const int b = item.x;
    const double2 ct = center[b];
    const double rt = rho[b];
    double cb[P];  // row `lane` of the binomial matrix, C(k + lane, lane)
#pragma unroll
    for (int k = 0; k < P; ++k) cb[k] = lane < P ? c_binom.d[k + lane][lane] : 0.0;
    double2 acc = make_double2(0.0, 0.0);
    double b0 = 0.0;  // log kernel: constant term
    const int32_t* wl = widx + woff[b];
    for (int j = item.y; j < item.z; ++j) {
        const int s = wl[j];
        const double2 cs = center[s];
        const double rs = rho[s];
        const double dx = ct.x - cs.x, dy = ct.y - cs.y;
        const double r2 = dx * dx + dy * dy;
        const double inv = 1.0 / r2;
        const double2 u = make_double2(dx * inv, -dy * inv);
        const double2 alpha = make_double2(rs * u.x, rs * u.y);
        const double2 beta = make_double2(-rt * u.x, -rt * u.y);
        const double2 a = lane < P ? M64[(size_t)s * PS + lane] : make_double2(0.0, 0.0);
        const double2 v = cmul(lane_pow(alpha, lane), a);
        double2 w = make_double2(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const double2 vk = shfl2(v, k);
            w.x = fma(cb[k], vk.x, w.x);
            w.y = fma(cb[k], vk.y, w.y);
        }
        acc = cfma(cmul(u, lane_pow(beta, lane)), w, acc);
        if constexpr (LOG) {
            double t = (lane >= 1 && lane < P) ? -v.x / (double)lane : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            b0 += fma(0.5 * log(r2), __shfl_sync(0xffffffffu, a.x, 0), t);
        }
    }
    double2* out = item.w < 0 ? Lm2l + (size_t)b * PS : part + (size_t)it * PS;
    if (lane < P) out[lane] = acc;
    if constexpr (LOG) {
        if (lane == 0) out[P] = make_double2(b0, 0.0);
    }
}

// Levels with at most this many shifts use the warp-per-shift kernels.
constexpr int kWarpShiftMax = 1024;  // measured against 4096 and 16384: 1024 fastest

// ------------------------------------------------------------- L2P + sum

// Near field of sorted point i: P2P wrote it directly when its leaf has one
// work item, else one partial sum per item, added here in item order.
template <typename C>
struct NearParts {
    const int2* leaf_items;  // per box: first P2P item, item count
    const int32_t* bstart;
    const C* part;           // partial sums, row stride TS
    int TS;
    // separate evaluation points: P2P writes the near field by slot offset within the leaf (slot_of[i] -
    // pslot[leaf]) at the leaf's sorted positions; nullptr when slots follow the sorted order
    const int32_t* slot_of = nullptr;
    const int32_t* pslot = nullptr;
};
template <typename C>
__device__ __forceinline__ C near_of(int i, int lf, const C* __restrict__ nearv, const NearParts<C>& np) {
    const int2 li = np.leaf_items[lf];
    const int t = np.slot_of != nullptr ? np.slot_of[i] - np.pslot[lf] : i - np.bstart[lf];
    if (li.y <= 1) return nearv[np.bstart[lf] + t];
    C s{};
    for (int q = 0; q < li.y; ++q) {
        const C v = np.part[(size_t)(li.x + q) * np.TS + t];
        s.x += v.x;
        s.y += v.y;
    }
    return s;
}

// Scaled offset w = (z - c_b) / rho_b of a point from box b (FP32 hi/lo coordinates).
__device__ __forceinline__ float2 scaled_offset(const float4 pt, const float4* __restrict__ chl,
                                                const float* __restrict__ rho32, int b) {
    const float4 c = chl[b];
    const float r = rho32[b];
    const float inv = r > 0.f ? 1.0f / r : 0.f;
    return make_float2(((pt.x - c.x) + (pt.z - c.z)) * inv, ((pt.y - c.y) + (pt.w - c.w)) * inv);
}

// sum_{l < p} b_l w^l by Horner.  The M2L sums of a box hold P terms whatever
// the requested order p <= P; the terms l >= p are left out (the L2L drops
// them in the same way).
template <int P>
__device__ __forceinline__ float2 horner_p(const float2* __restrict__ b, const float2 w, int p) {
    float2 v = P - 1 < p ? b[P - 1] : make_float2(0.f, 0.f);
#pragma unroll
    for (int l = P - 2; l >= 0; --l) v = cfma(v, w, l < p ? b[l] : make_float2(0.f, 0.f));
    return v;
}

// One thread per sorted point: far field by Horner from the leaf's local
// expansion, plus the near field, written to the caller's order.  A leaf of
// the deepest level (fold_par >= 0) has no shifted local of its own: its far
// field is the parent's local at the point plus its own M2L sum at the point,
// which is the value the shifted local would give (up to rounding).
template <int P>
__device__ __forceinline__ void d_l2p32(const int vbx, int n, const int32_t* __restrict__ leaf_of,
                                               const int32_t* __restrict__ fold_par, const int2* __restrict__ box_m2l,
                                               const float4* __restrict__ chl,
                                               const float* __restrict__ rho32, const float4* __restrict__ pos4,
                                               const float2* __restrict__ L32, const float2* __restrict__ Lm2l,
                                               const float2* __restrict__ nearv, const NearParts<float2> np,
                                               const int32_t* __restrict__ perm, float2* __restrict__ out, int p,
                                               int PS) {
    int i = vbx * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf_of[i];
    const float4 pt = pos4[i];
    const int par = fold_par[lf];
    float2 v;
    if (par >= 0) {
        v = horner_p<P>(L32 + (size_t)par * PS, scaled_offset(pt, chl, rho32, par), P);
        if (box_m2l[lf].y > 0) {
            const float2 o = horner_p<P>(Lm2l + (size_t)lf * PS, scaled_offset(pt, chl, rho32, lf), p);
            v.x += o.x;
            v.y += o.y;
        }
    } else {
        v = horner_p<P>(L32 + (size_t)lf * PS, scaled_offset(pt, chl, rho32, lf), P);
    }
    const float2 nv = near_of(i, lf, nearv, np);
    out[perm[i]] = make_float2(v.x + nv.x, v.y + nv.y);
}
template <int P>
__global__ void __launch_bounds__(256) k_l2p32(int n, const int32_t* __restrict__ leaf_of,
                                               const int32_t* __restrict__ fold_par, const int2* __restrict__ box_m2l,
                                               const float4* __restrict__ chl,
                                               const float* __restrict__ rho32, const float4* __restrict__ pos4,
                                               const float2* __restrict__ L32, const float2* __restrict__ Lm2l,
                                               const float2* __restrict__ nearv, const NearParts<float2> np,
                                               const int32_t* __restrict__ perm, float2* __restrict__ out, int p,
                                               int PS) { d_l2p32<P>(blockIdx.x, n, leaf_of, fold_par, box_m2l, chl, rho32, pos4, L32, Lm2l, nearv, np, perm, out, p, PS); }

template <int P>
__global__ void __launch_bounds__(256) k_l2p64(int n, const int32_t* __restrict__ leaf_of,
                                               const double2* __restrict__ center,
                                               const double* __restrict__ rho, const double2* __restrict__ pts,
                                               const double2* __restrict__ L64, const double2* __restrict__ nearv,
                                               const NearParts<double2> np, const int32_t* __restrict__ perm,
                                               double2* __restrict__ out, int PS) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf_of[i];
    const double2 c = center[lf];
    const double r = rho[lf];
    const double inv = r > 0.0 ? 1.0 / r : 0.0;
    const double2 pt = pts[i];
    const double2 w = make_double2((pt.x - c.x) * inv, (pt.y - c.y) * inv);
    const double2* Lb = L64 + (size_t)lf * PS;
    double2 v = Lb[P - 1];
#pragma unroll
    for (int l = P - 2; l >= 0; --l) v = cfma(v, w, Lb[l]);
    const double2 nv = near_of(i, lf, nearv, np);
    out[perm[i]] = make_double2(v.x + nv.x, v.y + nv.y);
}

// Logarithmic kernel: both real-strength sets (L0: Re Gamma, L1: Im Gamma) at
// once, F_s = b0_s + rho Re(w sum_m bt_m w^m / (m+1)) by Horner, plus the
// complex near field (Re: set 0, Im: set 1).
template <int P, typename T2, typename T>
__device__ __forceinline__ T log_local_eval(const T2* __restrict__ Lb, const T2 w, const T r) {
    T2 h;
    h.x = Lb[P - 1].x * (T)(1.0 / P);
    h.y = Lb[P - 1].y * (T)(1.0 / P);
#pragma unroll
    for (int l = P - 2; l >= 0; --l) {
        T2 c;
        c.x = Lb[l].x * (T)(1.0 / (l + 1));
        c.y = Lb[l].y * (T)(1.0 / (l + 1));
        h = cfma(h, w, c);
    }
    return Lb[P].x + r * (w.x * h.x - w.y * h.y);
}

// log_local_eval of a box's own M2L sum: terms m >= p left out (as in the L2L).
template <int P>
__device__ __forceinline__ float log_local_eval_p(const float2* __restrict__ Lb, const float2 w, const float r,
                                                  int p) {
    float2 h = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = P - 1; l >= 0; --l) {
        const float2 c = l < p ? make_float2(Lb[l].x * (1.0f / (l + 1)), Lb[l].y * (1.0f / (l + 1)))
                               : make_float2(0.f, 0.f);
        h = cfma(h, w, c);
    }
    return Lb[P].x + r * (w.x * h.x - w.y * h.y);
}

// Same fold of the deepest level's L2L as in k_l2p32.
template <int P>
__global__ void __launch_bounds__(256) k_l2p32_log(int n, const int32_t* __restrict__ leaf_of,
                                                   const int32_t* __restrict__ fold_par,
                                                   const int2* __restrict__ box_m2l, const float4* __restrict__ chl,
                                                   const float* __restrict__ rho32, const float4* __restrict__ pos4,
                                                   const float2* __restrict__ L0, const float2* __restrict__ L1,
                                                   const float2* __restrict__ M0, const float2* __restrict__ M1,
                                                   const float2* __restrict__ nearv, const NearParts<float2> np,
                                                   const int32_t* __restrict__ perm, float2* __restrict__ out, int p,
                                                   int PS) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf_of[i];
    const float4 pt = pos4[i];
    const int par = fold_par[lf];
    const int b = par >= 0 ? par : lf;
    const float2 w = scaled_offset(pt, chl, rho32, b);
    const float r = rho32[b];
    float f0 = log_local_eval<P>(L0 + (size_t)b * PS, w, r);
    float f1 = log_local_eval<P>(L1 + (size_t)b * PS, w, r);
    if (par >= 0 && box_m2l[lf].y > 0) {
        const float2 wl = scaled_offset(pt, chl, rho32, lf);
        const float rl = rho32[lf];
        f0 += log_local_eval_p<P>(M0 + (size_t)lf * PS, wl, rl, p);
        f1 += log_local_eval_p<P>(M1 + (size_t)lf * PS, wl, rl, p);
    }
    const float2 nv = near_of(i, lf, nearv, np);
    out[perm[i]] = make_float2(f0 + nv.x, f1 + nv.y);
}

template <int P>
__global__ void __launch_bounds__(256) k_l2p64_log(int n, const int32_t* __restrict__ leaf_of,
                                                   const double2* __restrict__ center,
                                                   const double* __restrict__ rho, const double2* __restrict__ pts,
                                                   const double2* __restrict__ L0, const double2* __restrict__ L1,
                                                   const double2* __restrict__ nearv, const NearParts<double2> np,
                                                   const int32_t* __restrict__ perm, double2* __restrict__ out,
                                                   int PS) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf_of[i];
    const double2 c = center[lf];
    const double r = rho[lf];
    const double inv = r > 0.0 ? 1.0 / r : 0.0;
    const double2 pt = pts[i];
    const double2 w = make_double2((pt.x - c.x) * inv, (pt.y - c.y) * inv);
    const double f0 = log_local_eval<P>(L0 + (size_t)lf * PS, w, r);
    const double f1 = log_local_eval<P>(L1 + (size_t)lf * PS, w, r);
    const double2 nv = near_of(i, lf, nearv, np);
    out[perm[i]] = make_double2(f0 + nv.x, f1 + nv.y);
}

// --------------------------------------------------------------------- P2P

// Pairwise terms Gamma_j/(z_i - z_j) = Gamma_j conj(d)/|d|^2, d = z_i - z_j.
constexpr int kP2PBlocksPerSM = 4;

__device__ __forceinline__ void p2p_interact64(const double2 t, const double2 s, const double2 g, double2& acc) {
    const double dx = t.x - s.x, dy = t.y - s.y;
    const double r2 = fma(dx, dx, dy * dy);
    const double inv = rcp_nr64(r2);  // coincident pair (z_j = z_i, r2 = 0): adds 0
    const double tr = fma(g.x, dx, g.y * dy);
    const double ti = fma(g.y, dx, -g.x * dy);
    acc.x = fma(tr, inv, acc.x);
    acc.y = fma(ti, inv, acc.y);
}

__device__ __forceinline__ void p2p_fast(const double2 t, const double2 s, const double2 g, double2& acc) {
    p2p_interact64(t, s, g, acc);
}

// Logarithmic kernel, FP64: Gamma_j ln|z_i - z_j| (complex Gamma on the real
// kernel); a coincident pair adds 0.  Zero-strength padding sources sit at a
// finite position (the origin) and add exactly 0.
__device__ __forceinline__ void p2p_log(const double2 t, const double2 s, const double2 g, double2& acc) {
    const double dx = t.x - s.x, dy = t.y - s.y;
    const double r2 = fma(dx, dx, dy * dy);
    const double lr = r2 > 0.0 ? 0.5 * log(r2) : 0.0;
    acc.x = fma(g.x, lr, acc.x);
    acc.y = fma(g.y, lr, acc.y);
}

template <bool LOG, typename V, typename C>
__device__ __forceinline__ void p2p_term(const V t, const V s, const C g, C& acc) {
    if constexpr (LOG) p2p_log(t, s, g, acc);
    else p2p_fast(t, s, g, acc);
}

// ---- P2P over the leaf slot layout ------------------------------------------
// One warp per work item (a target leaf and a run of its strong entries),
// fetched from an atomic counter.  Lane (tg, ss) owns targets tg, tg+LT, ...
// (TPL of them) and source slice ss of S = 32/LT.  Every leaf occupies `cap`
// consecutive slots whose tail is zero-strength padding, so a source step is
// "slot offset of the range + ss" with no per-lane bounds test: S consecutive
// slots make one coalesced load.  When cap == S (LONG false) one step covers a
// whole range and the loop walks two ranges per half-iteration from two
// register sets (A, B) that are reloaded in place, with the range offsets read
// one half-iteration before the loads that use them.  Entries past the item's
// end read the all-padding block at slot `pad`.  The layouts with LT = 2 hold
// leaves of at most 16 = S points, so cap == S; the others (LONG) take
// ceil(count/S) steps per range.  The S slice sums are added with shuffles.
constexpr int kP2PDWarps = 4;

template <typename V, typename C, int TPL, int LT, bool LOG>
__global__ void __launch_bounds__(kP2PDWarps * 32, sizeof(C) == 8 ? 5 : 1)
    k_p2p_slots(const int4* __restrict__ items, const unsigned long long* __restrict__ nitems,
                unsigned* __restrict__ next_item, const int32_t* __restrict__ bstart,
                const int32_t* __restrict__ bcount, const int32_t* __restrict__ pslot,
                const int32_t* __restrict__ soff, const int2* __restrict__ srng, const V* __restrict__ posp,
                const C* __restrict__ gamp, C* __restrict__ nearv, C* __restrict__ part, int TS, int pad,
                int per_warp, const int32_t* __restrict__ rows, const unsigned long long* __restrict__ nheavy,
                long long cap, const int32_t* __restrict__ tfirst) {
    constexpr int S = 32 / LT;
    constexpr bool LONG = LT > 2;
    const int lane = threadIdx.x & 31;
    const int tg = lane % LT, ss = lane / LT;
    const int nit = (int)*nitems;
    const unsigned long long nh = *nheavy;
    for (int done = 0; done < per_warp; ++done) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(next_item, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nit) break;
        it = p2p_row_item(it, rows, nh, cap);
        const int4 item = items[it];
        const int b = item.x;
        const int ts = bstart[b], tn = bcount[b], tb = pslot[b];
        const int2* rl = srng + soff[b];
        const int ke = item.z;
        for (int t0 = tfirst != nullptr ? tfirst[b] : 0; t0 < tn; t0 += TPL * LT) {
            V xt[TPL];
            C acc[TPL];
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
                const int idx = t0 + tg + u * LT;
                xt[u] = (idx < tn) ? posp[tb + idx] : V{};
                acc[u] = C{};
            }
            if constexpr (!LONG) {
                int k = item.y;
                int oa0 = (k < ke ? rl[k].x : pad) + ss;
                int oa1 = (k + 1 < ke ? rl[k + 1].x : pad) + ss;
                V sa0 = posp[oa0], sa1 = posp[oa1];
                C ga0 = gamp[oa0], ga1 = gamp[oa1];
                int ob0 = (k + 2 < ke ? rl[k + 2].x : pad) + ss;
                int ob1 = (k + 3 < ke ? rl[k + 3].x : pad) + ss;
                while (true) {
                    const V sb0 = posp[ob0], sb1 = posp[ob1];
                    const C gb0 = gamp[ob0], gb1 = gamp[ob1];
                    oa0 = (k + 4 < ke ? rl[k + 4].x : pad) + ss;
                    oa1 = (k + 5 < ke ? rl[k + 5].x : pad) + ss;
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], sa0, ga0, acc[u]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], sa1, ga1, acc[u]);
                    if (k + 2 >= ke) break;
                    sa0 = posp[oa0];
                    sa1 = posp[oa1];
                    ga0 = gamp[oa0];
                    ga1 = gamp[oa1];
                    ob0 = (k + 6 < ke ? rl[k + 6].x : pad) + ss;
                    ob1 = (k + 7 < ke ? rl[k + 7].x : pad) + ss;
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], sb0, gb0, acc[u]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], sb1, gb1, acc[u]);
                    k += 4;
                    if (k >= ke) break;
                }
            } else {
                for (int k = item.y; k < ke; ++k) {
                    const int2 r = rl[k];
                    const int o = r.x + ss;
                    int e = 0;
                    for (; e + S < r.y; e += 2 * S) {  // two steps, both inside the range's slots
                        const V s0 = posp[o + e], s1 = posp[o + e + S];
                        const C g0 = gamp[o + e], g1 = gamp[o + e + S];
#pragma unroll
                        for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], s0, g0, acc[u]);
#pragma unroll
                        for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], s1, g1, acc[u]);
                    }
                    if (e < r.y) {
                        const V s0 = posp[o + e];
                        const C g0 = gamp[o + e];
#pragma unroll
                        for (int u = 0; u < TPL; ++u) p2p_term<LOG>(xt[u], s0, g0, acc[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
                C tot = acc[u];
#pragma unroll
                for (int o = LT; o < 32; o <<= 1) {
                    tot.x += __shfl_xor_sync(0xffffffffu, tot.x, o);
                    tot.y += __shfl_xor_sync(0xffffffffu, tot.y, o);
                }
                const int idx = t0 + tg + u * LT;
                if (ss == 0 && idx < tn) {
                    if (item.w < 0) nearv[ts + idx] = tot;
                    else part[(size_t)it * TS + idx] = tot;
                }
            }
        }
    }
}

// ---- FP32 P2P with packed f32x2 arithmetic ----------------------------------
// Same work items and slot layout as above, but a lane takes a PAIR of source
// slots per step and every instruction is a 2-wide FP32 operation: one target
// (duplicated into both halves once per target tile) against two sources.
// Per pair of interactions: 14 f32x2 instructions and 2 reciprocals, half the
// FP32 instruction issue of one-interaction-per-instruction code.  Lane (tg, ss): targets tg,
// tg+LT, ... and pair slice ss of S = 32/LT; a step covers 2S slots.  Each
// packed accumulator holds two partial sums (even / odd source slots), added
// at the end before the shuffle reduction over slices.
// Two sources (packed) against one target: Gamma_j conj(d)/|d|^2 with
// d = z_t - z_j from the hi/lo coordinates (so that z_t - z_j keeps full FP32
// relative accuracy even for very close pairs).  The coincident-pair guard is
// folded into |d|^2 (+1e-37f): coincident points give d = 0 and add 0; pairs
// closer than ~1e-18 are below FP32 resolution anyway.  Zero-strength padding
// sources add exactly 0 (every factor is finite).
struct SrcPair {
    f2x x, y, xl, yl, gx, gy, ngx;
};
__device__ __forceinline__ SrcPair src_pair(const ulonglong2 a, const ulonglong2 b, const ulonglong2 g) {
    SrcPair s;
    s.x = a.x;
    s.y = a.y;
    s.xl = b.x;
    s.yl = b.y;
    s.gx = g.x;
    s.gy = g.y;
    s.ngx = f2mul(g.x, f2pk(-1.f, -1.f));
    return s;
}
__device__ __forceinline__ void p2p_pair(const f2x tx, const f2x ty, const f2x txl, const f2x tyl, const SrcPair& s,
                                         f2x& ax, f2x& ay) {
    const f2x dx = f2add(f2sub(tx, s.x), f2sub(txl, s.xl));
    const f2x dy = f2add(f2sub(ty, s.y), f2sub(tyl, s.yl));
    const f2x r2 = f2fma(dx, dx, f2fma(dy, dy, f2pk(1e-37f, 1e-37f)));
    float r0, r1;
    f2upk(r2, r0, r1);
    const f2x inv = f2pk(rcp_approx(r0), rcp_approx(r1));
    const f2x a = f2mul(dx, inv), b = f2mul(dy, inv);
    ax = f2fma(s.gx, a, f2fma(s.gy, b, ax));   // gx a + gy b
    ay = f2fma(s.gy, a, f2fma(s.ngx, b, ay));  // gy a - gx b
}

// Logarithmic kernel, two sources against one target: Gamma_j log2(|d|^2)
// (the factor ln(2)/2 is applied to the finished sums).  Pairs with |d|^2
// below the smallest normal FP32 number (coincident points, or closer than
// ~1e-19) add 0.
__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float log2_pos(float r2) {
    return r2 >= 1.17549435e-38f ? lg2_ftz(r2) : 0.f;  // normal inputs only: the ftz form suffices
}
__device__ __forceinline__ void p2p_pair_log(const f2x tx, const f2x ty, const f2x txl, const f2x tyl,
                                             const SrcPair& s, f2x& ax, f2x& ay) {
    const f2x dx = f2add(f2sub(tx, s.x), f2sub(txl, s.xl));
    const f2x dy = f2add(f2sub(ty, s.y), f2sub(tyl, s.yl));
    const f2x r2 = f2fma(dx, dx, f2mul(dy, dy));
    float r0, r1;
    f2upk(r2, r0, r1);
    const f2x lg = f2pk(log2_pos(r0), log2_pos(r1));
    ax = f2fma(s.gx, lg, ax);
    ay = f2fma(s.gy, lg, ay);
}
// Real strengths (every imaginary part zero): Gamma_j conj(d)/|d|^2 = s (dx, -dy)
// with s = Gamma_j/|d|^2, accumulated as (sum s dx, sum s dy); the sign of the
// second sum is applied to the finished sums.  11 FP32 lane slots per pair
// instead of 14.
__device__ __forceinline__ void p2p_pair_real(const f2x tx, const f2x ty, const f2x txl, const f2x tyl,
                                              const SrcPair& s, f2x& ax, f2x& ay) {
    const f2x dx = f2add(f2sub(tx, s.x), f2sub(txl, s.xl));
    const f2x dy = f2add(f2sub(ty, s.y), f2sub(tyl, s.yl));
    const f2x r2 = f2fma(dx, dx, f2fma(dy, dy, f2pk(1e-37f, 1e-37f)));
    float r0, r1;
    f2upk(r2, r0, r1);
    const f2x sc = f2mul(s.gx, f2pk(rcp_approx(r0), rcp_approx(r1)));
    ax = f2fma(sc, dx, ax);
    ay = f2fma(sc, dy, ay);
}
template <bool LOG, bool REAL = false>
__device__ __forceinline__ void p2p_pair_t(const f2x tx, const f2x ty, const f2x txl, const f2x tyl,
                                           const SrcPair& s, f2x& ax, f2x& ay) {
    if constexpr (LOG) p2p_pair_log(tx, ty, txl, tyl, s, ax, ay);
    else if constexpr (REAL) p2p_pair_real(tx, ty, txl, tyl, s, ax, ay);
    else p2p_pair(tx, ty, txl, tyl, s, ax, ay);
}
constexpr float kHalfLn2 = 0.34657359027997264f;  // ln(2)/2: log2(|d|^2) -> ln|d|

// Blocks per SM: 7 for TPL <= 4 (72 registers, no spills; measured against 4 (124
// registers), 5, 6 (80) and 8 (64, spills): 7 is the fastest), 2 for TPL = 8.
// One work item of the warp (its target leaf against a run of its strong list).
template <int TPL, int LT, bool LOG, bool REAL = false>
__device__ __forceinline__ void d_p2p_pairs_item(const int it, const int4* __restrict__ items,
                                                 const int32_t* __restrict__ bstart,
                                                 const int32_t* __restrict__ bcount, const int32_t* __restrict__ pslot,
                                                 const int32_t* __restrict__ soff, const int2* __restrict__ srng,
                                                 const ulonglong2* __restrict__ posq,
                                                 const ulonglong2* __restrict__ gamq, float2* __restrict__ nearv,
                                                 float2* __restrict__ part, int TS, int pad,
                                                 const int32_t* __restrict__ tfirst) {
    constexpr int S = 32 / LT;      // pair slices
    constexpr bool LONG = LT > 4;   // the LT = 4 layouts hold leaves of at most 16 = 2S slots
    const int lane = threadIdx.x & 31;
    const int tg = lane % LT, ss = lane / LT;
    const int4 item = items[it];
    const int b = item.x;
    const int ts = bstart[b], tn = bcount[b], tb = pslot[b];
    const int2* rl = srng + soff[b];
    const int ke = item.z;
    // targets: the leaf's slots [t_first, tn) (with separate evaluation points its evaluation points)
    for (int t0 = tfirst != nullptr ? tfirst[b] : 0; t0 < tn; t0 += TPL * LT) {
        f2x tx[TPL], ty[TPL], txl[TPL], tyl[TPL], ax[TPL], ay[TPL];
#pragma unroll
        for (int u = 0; u < TPL; ++u) {
            const int idx = t0 + tg + u * LT;
            float x = 0.f, y = 0.f, xl = 0.f, yl = 0.f;
            if (idx < tn) {
                const int sl = tb + idx;
                const float* f = reinterpret_cast<const float*>(posq) + 8 * (sl >> 1) + (sl & 1);
                x = f[0];
                y = f[2];
                xl = f[4];
                yl = f[6];
            }
            tx[u] = f2pk(x, x);
            ty[u] = f2pk(y, y);
            txl[u] = f2pk(xl, xl);
            tyl[u] = f2pk(yl, yl);
            ax[u] = 0ull;
            ay[u] = 0ull;
        }
        if constexpr (!LONG) {
            // slot-pair index of range k's slice ss (the padding block past the end)
#define FMM_PIDX(k) ((((k) < ke ? rl[(k)].x : pad) >> 1) + ss)
            int k = item.y;
            int oa0 = FMM_PIDX(k), oa1 = FMM_PIDX(k + 1);
            ulonglong2 pa0 = posq[2 * oa0], qa0 = posq[2 * oa0 + 1], ga0 = gamq[oa0];
            ulonglong2 pa1 = posq[2 * oa1], qa1 = posq[2 * oa1 + 1], ga1 = gamq[oa1];
            int ob0 = FMM_PIDX(k + 2), ob1 = FMM_PIDX(k + 3);
            while (true) {
                const ulonglong2 pb0 = posq[2 * ob0], qb0 = posq[2 * ob0 + 1], gb0 = gamq[ob0];
                const ulonglong2 pb1 = posq[2 * ob1], qb1 = posq[2 * ob1 + 1], gb1 = gamq[ob1];
                oa0 = FMM_PIDX(k + 4);
                oa1 = FMM_PIDX(k + 5);
                {
                    const SrcPair s0 = src_pair(pa0, qa0, ga0), s1 = src_pair(pa1, qa1, ga1);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s0, ax[u], ay[u]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s1, ax[u], ay[u]);
                }
                if (k + 2 >= ke) break;
                pa0 = posq[2 * oa0];
                qa0 = posq[2 * oa0 + 1];
                ga0 = gamq[oa0];
                pa1 = posq[2 * oa1];
                qa1 = posq[2 * oa1 + 1];
                ga1 = gamq[oa1];
                ob0 = FMM_PIDX(k + 6);
                ob1 = FMM_PIDX(k + 7);
                {
                    const SrcPair s0 = src_pair(pb0, qb0, gb0), s1 = src_pair(pb1, qb1, gb1);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s0, ax[u], ay[u]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s1, ax[u], ay[u]);
                }
                k += 4;
                if (k >= ke) break;
            }
#undef FMM_PIDX
        } else {
            for (int k = item.y; k < ke; ++k) {
                const int2 r = rl[k];
                const int o = (r.x >> 1) + ss;  // slot-pair index of this slice
                int e = 0;                      // slot-pair offset of the step
                for (; 2 * (e + S) < r.y; e += 2 * S) {  // two steps, both inside the range's slots
                    const SrcPair s0 = src_pair(posq[2 * (o + e)], posq[2 * (o + e) + 1], gamq[o + e]);
                    const SrcPair s1 =
                        src_pair(posq[2 * (o + e + S)], posq[2 * (o + e + S) + 1], gamq[o + e + S]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s0, ax[u], ay[u]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s1, ax[u], ay[u]);
                }
                if (2 * e < r.y) {
                    const SrcPair s0 = src_pair(posq[2 * (o + e)], posq[2 * (o + e) + 1], gamq[o + e]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) p2p_pair_t<LOG, REAL>(tx[u], ty[u], txl[u], tyl[u], s0, ax[u], ay[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < TPL; ++u) {
            float x0, x1, y0, y1;
            f2upk(ax[u], x0, x1);
            f2upk(ay[u], y0, y1);
            float2 tot = make_float2(x0 + x1, y0 + y1);
#pragma unroll
            for (int o = LT; o < 32; o <<= 1) {
                tot.x += __shfl_xor_sync(0xffffffffu, tot.x, o);
                tot.y += __shfl_xor_sync(0xffffffffu, tot.y, o);
            }
            if constexpr (LOG) {
                tot.x *= kHalfLn2;
                tot.y *= kHalfLn2;
            }
            if constexpr (REAL) tot.y = -tot.y;
            const int idx = t0 + tg + u * LT;
            if (ss == 0 && idx < tn) {
                if (item.w < 0) nearv[ts + idx] = tot;
                else part[(size_t)it * TS + idx] = tot;
            }
        }
    }
}

template <int TPL, int LT, bool LOG>
__global__ void __launch_bounds__(kP2PDWarps * 32, TPL > 4 ? 2 : 7)
    k_p2p_pairs(const int4* __restrict__ items, const unsigned long long* __restrict__ nitems,
                unsigned* __restrict__ next_item, const int32_t* __restrict__ bstart,
                const int32_t* __restrict__ bcount, const int32_t* __restrict__ pslot,
                const int32_t* __restrict__ soff, const int2* __restrict__ srng, const ulonglong2* __restrict__ posq,
                const ulonglong2* __restrict__ gamq, float2* __restrict__ nearv, float2* __restrict__ part, int TS,
                int pad, int per_warp, const int32_t* __restrict__ rows, const unsigned long long* __restrict__ nheavy,
                long long cap, const unsigned* __restrict__ cplx, const int32_t* __restrict__ tfirst) {
    const int lane = threadIdx.x & 31;
    const int nit = (int)*nitems;
    const unsigned long long nh = *nheavy;
    const bool real = !LOG && *cplx == 0u;  // the gather saw no nonzero imaginary part
    for (int done = 0; done < per_warp; ++done) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(next_item, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nit) break;
        it = p2p_row_item(it, rows, nh, cap);
        if (real)
            d_p2p_pairs_item<TPL, LT, LOG, !LOG>(it, items, bstart, bcount, pslot, soff, srng, posq, gamq, nearv,
                                                 part, TS, pad, tfirst);
        else
            d_p2p_pairs_item<TPL, LT, LOG>(it, items, bstart, bcount, pslot, soff, srng, posq, gamq, nearv, part, TS,
                                           pad, tfirst);
    }
}

// M2L sums of boxes whose weak list was split: one warp per box, lane = coefficient
// (lanes stride over the PS slots: PS exceeds 32 at p = 32, with the log kernel's
// constant term in slot 32).
template <typename C>
__device__ __forceinline__ void d_reduce_m2l(const int vbx, int nbox, const int2* __restrict__ box_m2l,
                                                    const C* __restrict__ part, int PS, C* __restrict__ Lm2l) {
    const int b = (int)((vbx * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nbox) return;
    const int2 mi = box_m2l[b];
    if (mi.y <= 1) return;
    for (int c = lane; c < PS; c += 32) {
        C s{};
#pragma unroll 8
        for (int q = 0; q < mi.y; ++q) {
            const C v = part[(size_t)(mi.x + q) * PS + c];
            s.x += v.x;
            s.y += v.y;
        }
        Lm2l[(size_t)b * PS + c] = s;
    }
}
template <typename C>
__global__ void __launch_bounds__(256) k_reduce_m2l(int nbox, const int2* __restrict__ box_m2l,
                                                    const C* __restrict__ part, int PS, C* __restrict__ Lm2l) { d_reduce_m2l<C>(blockIdx.x, nbox, box_m2l, part, PS, Lm2l); }

// Diagnostic: the P2P's FP64 reciprocal over an array (tests compare it with
// the correctly rounded 1/x).
__global__ void k_selftest_rcp64(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = rcp_nr64(x[i]);
}
void launch_selftest_rcp64(const double* x, int64_t n, double* out, cudaStream_t s) {
    k_selftest_rcp64<<<nblk(n, 256), 256, 0, s>>>(x, n, out);
}

// ================================================= persistent evaluation
// FMM_FLAG_PERSISTENT (FP32 path, harmonic kernel): the whole evaluation of a
// tree -- one instance or a forest of many -- in ONE launch.  Its CTAs take
// units from a device work queue: an atomic ticket counter runs over a table
// of stages, each stage a range of virtual blocks of 128 threads that run the
// body of one of the pass kernels above (the same arithmetic in the same
// order per box, item and point).  Before a unit runs, its CTA waits, with a
// bounded spin, until the units its stage depends on are complete: a
// far-field stage waits for every far-field unit before it (the strengths for
// P2M, the level below for M2M, the whole upward pass for M2L, the level above
// for L2L), P2P units only for the strength gather, L2P for everything.  A
// unit waits only on units with smaller tickets, which running CTAs already
// hold, so the queue always advances.  P2P units are interleaved between the
// far-field stages, so that CTAs that wait on a level of the far field have
// P2P work behind them.  M2L runs on the CUDA cores (the body of k_m2l32): the
// tensor-core M2L wants whole CTAs with 168 registers and its tensor memory.
enum : int { PT_GATHER = 0, PT_P2M_T, PT_P2M_W, PT_M2M_T, PT_M2M_W, PT_M2L, PT_REDUCE, PT_L2L_T, PT_L2L_W, PT_P2P,
             PT_L2P };

struct PStage {
    long long ticket0;   // first ticket of the stage
    long long need_far;  // far-field units that must be complete before a unit of the stage runs
    long long need_p2p;  // P2P units that must be complete
    const int32_t* ids;  // the stage's box list (leaves, a level's parents or boxes)
    int type;
    int nvb;             // virtual blocks (units) of the stage
    int vb0;             // first virtual block of the stage within its pass (P2P is cut into chunks)
    int cnt;             // entries of `ids`
    int arg;             // P2M: write the FP64 copy (parents); L2L: FP32 copy of every box (all32)
    int pad_;
};
constexpr int kMaxPStages = 96;

struct PArgs {
    const PStage* st;
    int nst;
    long long total;
    unsigned long long* ctr;  // [0] ticket, [1] far-field units done, [2] P2P units done
    unsigned* status;
    unsigned* cplx;              // set by the gather units when a strength has a nonzero imaginary part
    unsigned long long wait_ns;  // bound of one queue wait
    int n, nbox, p, PS, lay, pad, TS;
    const double2* gin;
    const int32_t *perm, *slot_of, *bstart, *bcount, *child0, *parent, *leaf_of, *fold_par, *pslot, *soff, *woff,
        *widx, *m2l_rows;
    const float4 *chl, *pos4;
    const float* rho32;
    const double* rho;
    const double2* center;
    const int2 *box_m2l, *srng, *leaf_items;
    const int4 *m2l_items, *p2p_items;
    const unsigned long long *n_m2l, *n_p2p, *p2p_nheavy;
    const int32_t* p2p_rows;
    long long p2p_cap;
    const int32_t* tfirst;     // separate evaluation points: per leaf the first target slot (nullptr otherwise)
    const int32_t* near_slot;  // separate evaluation points: slot of every sorted position (nullptr otherwise)
    const ulonglong2* posq;
    float2* gam;
    float* gamp;
    float2 *M32, *Lm2l, *m2l_part, *L32, *nearv, *p2p_part, *out;
    double2 *M64, *L64;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until at least need_far far-field units and need_p2p P2P units are
// complete.  Bounded in time (limit_ns of the GPU's global timer, whatever the
// sleeps between polls actually last): on expiry it sets ST_TIMEOUT, records
// the waiting stage (+1) in ctr[3] and returns false.
__device__ bool pq_wait(unsigned long long* ctr, long long need_far, long long need_p2p, unsigned* status,
                        unsigned long long limit_ns, int stage) {
    const unsigned long long t0 = global_ns();
    while (true) {
        if ((long long)ld_acquire_u64(ctr + 1) >= need_far && (long long)ld_acquire_u64(ctr + 2) >= need_p2p)
            return true;
        if (global_ns() - t0 > limit_ns) {
            atomicOr(status, ST_TIMEOUT);
            atomicMax(ctr + 3, (unsigned long long)(stage + 1));
            return false;
        }
        __nanosleep(128);
    }
}

// Self-test of the queue's bounded wait: a unit that needs one far-field unit
// more than will ever complete must give up (after `limit_ns`) and report
// ST_TIMEOUT.
__global__ void k_selftest_queue(unsigned long long* ctr, unsigned long long limit_ns, unsigned* status) {
    if (threadIdx.x == 0) pq_wait(ctr, (long long)ld_acquire_u64(ctr + 1) + 1, 0, status, limit_ns, 0);
}
void launch_selftest_queue(unsigned long long* ctr, unsigned long long limit_ns, unsigned* status, cudaStream_t s) {
    k_selftest_queue<<<1, 32, 0, s>>>(ctr, limit_ns, status);
}

// P2P units run after the gather stage, so the complex-strength flag is final: the real form when it is clear.
template <int TPL, int LT>
__device__ __forceinline__ void pq_p2p(const PArgs& a, int it) {
    const ulonglong2* gq = reinterpret_cast<const ulonglong2*>(a.gamp);
    if (*reinterpret_cast<volatile const unsigned*>(a.cplx) == 0u)
        d_p2p_pairs_item<TPL, LT, false, true>(it, a.p2p_items, a.bstart, a.bcount, a.pslot, a.soff, a.srng, a.posq,
                                               gq, a.nearv, a.p2p_part, a.TS, a.pad, a.tfirst);
    else
        d_p2p_pairs_item<TPL, LT, false>(it, a.p2p_items, a.bstart, a.bcount, a.pslot, a.soff, a.srng, a.posq, gq,
                                         a.nearv, a.p2p_part, a.TS, a.pad, a.tfirst);
}

template <int P>
__device__ __forceinline__ void pq_unit(const PArgs& a, const PStage& g, int vb) {
    switch (g.type) {
        case PT_GATHER:  // also flags complex strengths (the whole CTA runs the unit: its block-wide OR is safe)
            d_gather32(vb, a.gin, a.perm, a.slot_of, a.n, a.gam, a.gamp, a.cplx);
            break;
        case PT_P2M_T:
            d_p2m32<P>(vb, g.ids, g.cnt, a.bstart, a.bcount, a.chl, a.rho32, a.pos4, a.gam, a.M32,
                       g.arg ? a.M64 : nullptr, a.p, a.PS);
            break;
        case PT_P2M_W:
            d_p2m32_warp<P>(vb, g.ids, g.cnt, a.bstart, a.bcount, a.chl, a.rho32, a.pos4, a.gam, a.M32, a.M64, a.p,
                            a.PS);
            break;
        case PT_M2M_T:
            d_m2m<P>(vb, g.ids, g.cnt, a.child0, a.rho, a.center, a.M32, a.M64, a.M32, 1, a.p, a.PS);
            break;
        case PT_M2M_W:
            d_m2m_warp<P>(vb, g.ids, g.cnt, a.child0, a.rho, a.center, a.M32, a.M64, a.M32, 1, a.p, a.PS);
            break;
        case PT_M2L:
            d_m2l32<P, false>(vb, a.m2l_items, a.n_m2l, a.woff, a.widx, a.chl, a.rho32, a.M32, a.Lm2l, a.m2l_part,
                              a.m2l_rows, a.PS);
            break;
        case PT_REDUCE:
            d_reduce_m2l<float2>(vb, a.nbox, a.box_m2l, a.m2l_part, a.PS, a.Lm2l);
            break;
        case PT_L2L_T:
            d_l2l<P, float2, false>(vb, g.ids, g.cnt, a.parent, a.child0, a.rho, a.center, a.box_m2l, a.Lm2l, a.L64,
                                    a.L32, g.arg, a.p, a.PS);
            break;
        case PT_L2L_W:
            d_l2l_warp<P, float2, false>(vb, g.ids, g.cnt, a.parent, a.child0, a.rho, a.center, a.box_m2l, a.Lm2l,
                                         a.L64, a.L32, g.arg, a.p, a.PS);
            break;
        case PT_P2P: {
            int it = vb * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);  // one item per warp, in row order
            if (it < (int)*a.n_p2p) {
                it = p2p_row_item(it, a.p2p_rows, *a.p2p_nheavy, a.p2p_cap);
                switch (a.lay) {
                    case 204: pq_p2p<2, 4>(a, it); break;
                    case 404: pq_p2p<4, 4>(a, it); break;
                    case 408: pq_p2p<4, 8>(a, it); break;
                    case 416: pq_p2p<4, 16>(a, it); break;
                    default: pq_p2p<8, 16>(a, it); break;
                }
            }
            break;
        }
        case PT_L2P: {
            const NearParts<float2> np{a.leaf_items, a.bstart, a.p2p_part, a.TS, a.near_slot, a.pslot};
            d_l2p32<P>(vb, a.n, a.leaf_of, a.fold_par, a.box_m2l, a.chl, a.rho32, a.pos4, a.L32, a.Lm2l, a.nearv, np,
                       a.perm, a.out, a.p, a.PS);
            break;
        }
    }
}

// The persistent kernel: a CTA takes the next ticket, finds its stage (the
// table is copied to shared memory once), waits for the stage's dependencies,
// runs the unit, and counts it as complete (fence, then one atomic).  A CTA
// whose wait gave up stops taking tickets (ST_TIMEOUT is set; the units that
// depend on it give up the same way).
template <int P>
__global__ void __launch_bounds__(128, 4) k_eval_persistent(const PArgs a) {
    __shared__ PStage sst[kMaxPStages];
    __shared__ int s_stage, s_vb, s_go;
    for (int i = threadIdx.x; i < a.nst; i += blockDim.x) sst[i] = a.st[i];
    __syncthreads();
    // a CTA can take at most every ticket: more rounds than that mean a broken table (reported, not looped)
    for (long long round = 0;; ++round) {
        if (round > a.total) {
            if (threadIdx.x == 0) atomicOr(a.status, ST_INTERNAL);
            break;
        }
        if (threadIdx.x == 0) {
            const long long tk = (long long)atomicAdd(a.ctr, 1ull);
            int go = 0, g = 0;
            if (tk < a.total) {
                while (g + 1 < a.nst && sst[g + 1].ticket0 <= tk) ++g;
                go = pq_wait(a.ctr, sst[g].need_far, sst[g].need_p2p, a.status, a.wait_ns, g) ? 1 : 0;
                __threadfence();
            }
            s_stage = g;
            s_vb = go ? sst[g].vb0 + (int)(tk - sst[g].ticket0) : 0;
            s_go = go;
        }
        __syncthreads();
        const int go = s_go, g = s_stage, vb = s_vb;
        if (!go) break;
        pq_unit<P>(a, sst[g], vb);
        __syncthreads();  // the unit's writes are done (and s_* may be overwritten)
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.ctr + (sst[g].type == PT_P2P ? 2 : 1), 1ull);
        }
    }
}
// ============================================================ dispatch

Bufs bufs(Tree& t, int set) {
    const size_t nb = (size_t)t.nbox, n = (size_t)t.n, PS = (size_t)t.PS;
    const size_t cs = t.path == FMM_PATH_FP32 ? sizeof(float2) : sizeof(double2);
    Bufs b;
    b.gam = static_cast<char*>(t.d_gam) + set * n * cs;
    b.near = t.d_near;
    b.M64 = t.d_M64 + set * nb * PS;
    b.M32 = t.d_M32 + set * nb * PS;
    b.L64 = t.d_L64 + set * nb * PS;
    b.L32 = t.d_L32 + set * nb * PS;
    b.Lm2l = static_cast<char*>(t.d_Lm2l) + set * nb * PS * cs;
    b.p2p_part = t.d_p2p_part;
    b.m2l_part = static_cast<char*>(t.d_m2l_part) + set * (size_t)t.part_m2l_cap * PS * cs;
    return b;
}

// Launch grids cover the last build's work-item counts plus 25 % slack (the
// kernels read the exact count on the device), not the allocated capacities,
// which can stay far larger after a build at another N_levels.
static long long grid_target(unsigned long long c) { return (long long)(c + c / 4 + 64); }
bool refresh_grids(Tree& t) {
    bool changed = false;
    const long long cp = (long long)t.h_counts[2], cm = (long long)t.h_counts[3];
    if (t.grid_p2p_items < cp || t.grid_p2p_items > 5 * (cp + 64) / 2) {
        t.grid_p2p_items = std::min(grid_target(cp), std::max(t.p2p_cap, 1LL));
        changed = true;
    }
    if (t.grid_m2l_items < cm || t.grid_m2l_items > 5 * (cm + 64) / 2) {
        t.grid_m2l_items = std::min(grid_target(cm), std::max(t.m2l_cap, 1LL));
        changed = true;
    }
    return changed;
}
long long p2p_grid_items(const Tree& t) { return t.grid_p2p_items > 0 ? t.grid_p2p_items : t.p2p_cap; }
long long m2l_grid_items(const Tree& t) { return t.grid_m2l_items > 0 ? t.grid_m2l_items : t.m2l_cap; }

static const unsigned long long* item_count(const Tree& t, int which) {
    return reinterpret_cast<const unsigned long long*>(t.d_status) + 1 + which;  // 2 = P2P, 3 = M2L
}

// Upward pass (P2M, M2M): needs the tree, not the coupling lists.
template <int P>
static void launch_up_fp32(Tree& t, const Bufs& B, cudaStream_t s) {
    const float2* gam = static_cast<const float2*>(B.gam);
    k_p2m32<P><<<nblk(t.nleaf, 128), 128, 0, s>>>(t.leaves.d_ids, (int)t.nleaf, t.d_bstart, t.d_bcount, t.d_chl,
                                                  t.d_rho32, t.d_pos4, gam, B.M32, nullptr, t.p, t.PS);
    // parent levels whose boxes hold few points take their multipoles from their points (p2m_parent_mode):
    // up to 64 points a thread per box, up to 1024 a warp per box; the levels above them shift in FP64
    for (int l = t.Lmax - 2; l >= 0; --l) {
        const LevelList& L = t.level_parents[l];
        if (!L.count) continue;
        const int how = p2m_parent_mode(t, l);
        if (how == 1)
            k_p2m32<P><<<nblk(L.count, 128), 128, 0, s>>>(L.d_ids, L.count, t.d_bstart, t.d_bcount, t.d_chl,
                                                          t.d_rho32, t.d_pos4, gam, B.M32, B.M64, t.p, t.PS);
        else if (how == 2)
            k_p2m32_warp<P><<<nblk(32 * (int64_t)L.count, 128), 128, 0, s>>>(L.d_ids, L.count, t.d_bstart,
                                                                             t.d_bcount, t.d_chl, t.d_rho32,
                                                                             t.d_pos4, gam, B.M32, B.M64, t.p, t.PS);
    }
    for (int l = t.Lmax - 2; l >= 0; --l) {
        const LevelList& L = t.level_parents[l];
        if (!L.count || p2m_parent_mode(t, l) != 0) continue;
        if (4 * (int64_t)L.count <= kWarpShiftMax)
            k_m2m_warp<P><<<L.count, 128, 0, s>>>(L.d_ids, L.count, t.d_child0, t.d_rho, t.d_center, B.M32, B.M64,
                                                  B.M32, 1, t.p, t.PS);
        else
            k_m2m<P><<<nblk(4 * (int64_t)L.count, 128), 128, 0, s>>>(L.d_ids, L.count, t.d_child0, t.d_rho,
                                                                     t.d_center, B.M32, B.M64, B.M32, 1, t.p, t.PS);
    }
}

// Downward pass (M2L, ordered M2L sums, L2L): needs the lists.
template <int P, bool LOG>
static void launch_down_fp32(Tree& t, const Bufs& B, cudaStream_t s) {
    if (t.flags & FMM_FLAG_TIMING) cudaEventRecord(t.ev_t[2], s);
    if (m2l_tc_enabled()) {
        launch_m2l_tc(t, B.M32, static_cast<float2*>(B.Lm2l), static_cast<float2*>(B.m2l_part), LOG, s);
        k_reduce_m2l<float2><<<nblk(32 * t.nbox, 256), 256, 0, s>>>((int)t.nbox, t.d_box_m2l,
                                                                   static_cast<const float2*>(B.m2l_part), t.PS,
                                                                   static_cast<float2*>(B.Lm2l));
    } else {
        k_m2l32<P, LOG><<<nblk(m2l_grid_items(t), 128), 128, 0, s>>>(t.d_m2l_items, item_count(t, 3), t.d_woff, t.d_widx,
                                                        t.d_chl, t.d_rho32, B.M32, static_cast<float2*>(B.Lm2l),
                                                        static_cast<float2*>(B.m2l_part), t.d_m2l_rows, t.PS);
        k_reduce_m2l<float2><<<nblk(32 * t.nbox, 256), 256, 0, s>>>((int)t.nbox, t.d_box_m2l,
                                                                   static_cast<const float2*>(B.m2l_part), t.PS,
                                                                   static_cast<float2*>(B.Lm2l));
    }
    if (t.flags & FMM_FLAG_TIMING) cudaEventRecord(t.ev_t[3], s);
    // the deepest level's leaves get no L2L (see fold_leaf_l2l); the level above then keeps an FP32 copy
    // of every box's local for their L2P
    const bool fold = fold_leaf_l2l(t);
    const int lend = fold ? t.Lmax - 2 : t.Lmax - 1;  // deepest level that gets an L2L
    for (int l = 0; l + 1 <= lend; ++l) {
        const LevelList& L = t.level_boxes[l + 1];
        const int all32 = fold && l + 1 == lend;
        if (L.count <= kWarpShiftMax)
            k_l2l_warp<P, float2, LOG><<<nblk(32 * (int64_t)L.count, 128), 128, 0, s>>>(
                L.d_ids, L.count, t.d_parent, t.d_child0, t.d_rho, t.d_center, t.d_box_m2l,
                static_cast<const float2*>(B.Lm2l), B.L64, B.L32, all32, t.p, t.PS);
        else
            k_l2l<P, float2, LOG><<<nblk(L.count, 128), 128, 0, s>>>(
                L.d_ids, L.count, t.d_parent, t.d_child0, t.d_rho, t.d_center, t.d_box_m2l,
                static_cast<const float2*>(B.Lm2l), B.L64, B.L32, all32, t.p, t.PS);
    }
}

template <int P>
static void launch_up_fp64(Tree& t, const Bufs& B, cudaStream_t s) {
    const double2* gam = static_cast<const double2*>(B.gam);
    k_p2m64<P><<<nblk(t.nleaf, 128), 128, 0, s>>>(t.leaves.d_ids, (int)t.nleaf, t.d_bstart, t.d_bcount, t.d_center,
                                                  t.d_rho, t.d_pts, gam, B.M64, t.p, t.PS);
    for (int l = t.Lmax - 2; l >= 0; --l) {
        const LevelList& L = t.level_parents[l];
        if (!L.count) continue;
        if (4 * (int64_t)L.count <= kWarpShiftMax)
            k_m2m_warp<P><<<L.count, 128, 0, s>>>(L.d_ids, L.count, t.d_child0, t.d_rho, t.d_center, nullptr,
                                                  B.M64, nullptr, 0, t.p, t.PS);
        else
            k_m2m<P><<<nblk(4 * (int64_t)L.count, 128), 128, 0, s>>>(L.d_ids, L.count, t.d_child0, t.d_rho,
                                                                     t.d_center, nullptr, B.M64, nullptr, 0, t.p,
                                                                     t.PS);
    }
}

template <int P, bool LOG>
static void launch_down_fp64(Tree& t, const Bufs& B, cudaStream_t s) {
    if (t.flags & FMM_FLAG_TIMING) cudaEventRecord(t.ev_t[2], s);
    if (m2l_grid_items(t) <= 64LL * t.num_sms)  // few items: a warp per item (lane = output coefficient)
        k_m2l64_warp<P, LOG><<<nblk(32 * m2l_grid_items(t), 128), 128, 0, s>>>(
            t.d_m2l_items, item_count(t, 3), t.d_woff, t.d_widx, t.d_center, t.d_rho, B.M64,
            static_cast<double2*>(B.Lm2l), static_cast<double2*>(B.m2l_part), t.d_m2l_rows, t.PS);
    else
        k_m2l64<P, LOG><<<nblk(m2l_grid_items(t), 128), 128, 0, s>>>(t.d_m2l_items, item_count(t, 3), t.d_woff, t.d_widx,
                                                        t.d_center, t.d_rho, B.M64, static_cast<double2*>(B.Lm2l),
                                                        static_cast<double2*>(B.m2l_part), t.d_m2l_rows, t.PS);
    k_reduce_m2l<double2><<<nblk(32 * t.nbox, 256), 256, 0, s>>>((int)t.nbox, t.d_box_m2l,
                                                                static_cast<const double2*>(B.m2l_part), t.PS,
                                                                static_cast<double2*>(B.Lm2l));
    if (t.flags & FMM_FLAG_TIMING) cudaEventRecord(t.ev_t[3], s);
    for (int l = 0; l + 1 < t.Lmax; ++l) {
        const LevelList& L = t.level_boxes[l + 1];
        if (L.count <= kWarpShiftMax)
            k_l2l_warp<P, double2, LOG><<<nblk(32 * (int64_t)L.count, 128), 128, 0, s>>>(
                L.d_ids, L.count, t.d_parent, t.d_child0, t.d_rho, t.d_center, t.d_box_m2l,
                static_cast<const double2*>(B.Lm2l), B.L64, nullptr, 0, t.p, t.PS);
        else
            k_l2l<P, double2, LOG><<<nblk(L.count, 128), 128, 0, s>>>(
                L.d_ids, L.count, t.d_parent, t.d_child0, t.d_rho, t.d_center, t.d_box_m2l,
                static_cast<const double2*>(B.Lm2l), B.L64, nullptr, 0, t.p, t.PS);
    }
}

template <typename C>
static NearParts<C> near_parts(const Tree& t, const Bufs& B) {
    return NearParts<C>{t.d_leaf_items, t.d_bstart, static_cast<const C*>(B.p2p_part), t.max_leaf,
                        t.n_src > 0 ? t.d_slot_of : nullptr, t.n_src > 0 ? t.d_pslot : nullptr};
}

template <int P>
static void launch_l2p(Tree& t, const Bufs& B, void* d_phi, cudaStream_t s) {
    const int n = (int)t.n;
    if (t.path == FMM_PATH_FP32) {
        k_l2p32<P><<<nblk(n, 256), 256, 0, s>>>(n, t.d_leaf_of, t.d_fold_par, t.d_box_m2l, t.d_chl, t.d_rho32,
                                                t.d_pos4, B.L32, static_cast<const float2*>(B.Lm2l),
                                                static_cast<const float2*>(B.near), near_parts<float2>(t, B), t.d_perm,
                                                static_cast<float2*>(d_phi), t.p, t.PS);
    } else {
        k_l2p64<P><<<nblk(n, 256), 256, 0, s>>>(n, t.d_leaf_of, t.d_center, t.d_rho, t.d_pts, B.L64,
                                                static_cast<const double2*>(B.near), near_parts<double2>(t, B),
                                                t.d_perm, static_cast<double2*>(d_phi), t.PS);
    }
}

template <int P>
static void launch_l2p_log(Tree& t, const Bufs& B0, const Bufs& B1, void* d_phi, cudaStream_t s) {
    const int n = (int)t.n;
    if (t.path == FMM_PATH_FP32) {
        k_l2p32_log<P><<<nblk(n, 256), 256, 0, s>>>(
            n, t.d_leaf_of, t.d_fold_par, t.d_box_m2l, t.d_chl, t.d_rho32, t.d_pos4, B0.L32, B1.L32,
            static_cast<const float2*>(B0.Lm2l), static_cast<const float2*>(B1.Lm2l),
            static_cast<const float2*>(B0.near), near_parts<float2>(t, B0), t.d_perm, static_cast<float2*>(d_phi), t.p,
            t.PS);
    } else {
        k_l2p64_log<P><<<nblk(n, 256), 256, 0, s>>>(n, t.d_leaf_of, t.d_center, t.d_rho, t.d_pts, B0.L64, B1.L64,
                                                    static_cast<const double2*>(B0.near), near_parts<double2>(t, B0),
                                                    t.d_perm, static_cast<double2*>(d_phi), t.PS);
    }
}

// Work items one P2P warp takes before it exits (FMM_P2P_ITEMS_PER_WARP
// overrides; 0 = persistent grid of FMM_P2P_BLOCKS_PER_SM blocks per SM).
// Bounded warps let blocks retire during the pass, so the far-field kernels
// on the high-priority stream get SM slots while P2P runs.  Measured on the
// 1e6-point workload: items of up to 4096 sources, one per warp, beat items of
// 2048 sources four per warp (fewer split leaves, so fewer partial sums;
// evaluation 2.16 -> 2.11 ms) and items of 8192 sources.
constexpr int kP2PItemsPerWarp = 1;
static int env_int(const char* name, int dflt) {
    const char* e = getenv(name);
    return e ? atoi(e) : dflt;
}
static int p2p_items_per_warp() {
    static int v = env_int("FMM_P2P_ITEMS_PER_WARP", kP2PItemsPerWarp);
    return v;
}
static int p2p_blocks_per_sm() {
    static int v = [] {
        const int x = env_int("FMM_P2P_BLOCKS_PER_SM", 0);
        return x > 0 ? x : kP2PBlocksPerSM;
    }();
    return v;
}

template <bool LOG>
static void launch_p2p(Tree& t, const Bufs& B, cudaStream_t s) {
    const unsigned long long* cnt = item_count(t, 2);
    unsigned* next = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned long long*>(t.d_status) + 7);
    cudaMemsetAsync(next, 0, sizeof(unsigned), s);
    int per_warp = p2p_items_per_warp();
    int dgrid;
    if (per_warp > 0) {
        dgrid = nblk(p2p_grid_items(t), kP2PDWarps * per_warp);
    } else {
        per_warp = 1 << 30;
        dgrid = std::min(nblk(p2p_grid_items(t), kP2PDWarps), t.num_sms * p2p_blocks_per_sm());
    }
    const P2PLayout lay = p2p_layout(t.max_leaf);
    const int pad = (int)(t.nleaf * t.leaf_cap);
    const unsigned long long* nheavy = t.d_m2l_rowctr + kM2LItemPairsMax + 1;
    const int32_t* tfirst = t.n_src > 0 ? t.d_nsrc : nullptr;  // separate evaluation points: targets only
#define FMM_P2P(V, C, TPL, LT)                                                                                   \
    t.p2p_funcs.push_back(reinterpret_cast<const void*>(k_p2p_slots<V, C, TPL, LT, LOG>));                      \
    k_p2p_slots<V, C, TPL, LT, LOG><<<dgrid, kP2PDWarps * 32, 0, s>>>(                                            \
        t.d_p2p_items, cnt, next, t.d_bstart, t.d_bcount, t.d_pslot, t.d_soff, t.d_srng,                          \
        static_cast<const V*>(t.d_posp), static_cast<const C*>(t.d_gamp), nv, pt, t.max_leaf, pad, per_warp,      \
        t.d_p2p_rows, nheavy, t.p2p_cap, tfirst);
#define FMM_P2P_LAYOUTS(V, C)                                  \
    switch (lay.tpl * 100 + lay.lt) {                          \
        case 202: FMM_P2P(V, C, 2, 2) break;                   \
        case 402: FMM_P2P(V, C, 4, 2) break;                   \
        case 802: FMM_P2P(V, C, 8, 2) break;                   \
        case 804: FMM_P2P(V, C, 8, 4) break;                   \
        case 808: FMM_P2P(V, C, 8, 8) break;                   \
        default: FMM_P2P(V, C, 8, 16) break;                   \
    }
    if (t.path == FMM_PATH_FP32) {
        float2* nv = static_cast<float2*>(B.near);
        float2* pt = static_cast<float2*>(B.p2p_part);
        const P2PLayout pl = p2p_pair_layout(t.max_leaf);
#define FMM_P2P_PAIRS(TPL, LT)                                                                                   \
    t.p2p_funcs.push_back(reinterpret_cast<const void*>(k_p2p_pairs<TPL, LT, LOG>));                            \
    k_p2p_pairs<TPL, LT, LOG><<<dgrid, kP2PDWarps * 32, 0, s>>>(                                                  \
        t.d_p2p_items, cnt, next, t.d_bstart, t.d_bcount, t.d_pslot, t.d_soff, t.d_srng,                          \
        static_cast<const ulonglong2*>(t.d_posp), static_cast<const ulonglong2*>(t.d_gamp), nv, pt, t.max_leaf,   \
        pad, per_warp, t.d_p2p_rows, nheavy, t.p2p_cap, t.d_status + 1, tfirst);
        switch (pl.tpl * 100 + pl.lt) {
            case 204: FMM_P2P_PAIRS(2, 4) break;
            case 404: FMM_P2P_PAIRS(4, 4) break;
            case 408: FMM_P2P_PAIRS(4, 8) break;
            case 416: FMM_P2P_PAIRS(4, 16) break;
            default: FMM_P2P_PAIRS(8, 16) break;
        }
#undef FMM_P2P_PAIRS
    } else {
        double2* nv = static_cast<double2*>(B.near);
        double2* pt = static_cast<double2*>(B.p2p_part);
        FMM_P2P_LAYOUTS(double2, double2)
    }
#undef FMM_P2P_LAYOUTS
#undef FMM_P2P
}

template <int P>
static void launch_up(Tree& t, const Bufs& B, cudaStream_t s) {
    if (t.path == FMM_PATH_FP32) launch_up_fp32<P>(t, B, s);
    else launch_up_fp64<P>(t, B, s);
}
template <int P, bool LOG>
static void launch_down(Tree& t, const Bufs& B, cudaStream_t s) {
    if (t.path == FMM_PATH_FP32) launch_down_fp32<P, LOG>(t, B, s);
    else launch_down_fp64<P, LOG>(t, B, s);
}

// Compiled expansion orders; a request for p runs the smallest compiled
// order >= p with the coefficients k >= p held at zero.
#define FMM_FOR_ORDERS(X) X(4) X(8) X(12) X(16) X(17) X(20) X(24) X(28) X(32)

int compiled_order(int p) {
#define FMM_PICK(Q) \
    if (p <= Q) return Q;
    FMM_FOR_ORDERS(FMM_PICK)
#undef FMM_PICK
    return -1;
}

void dispatch_up(Tree& t, const Bufs& B, cudaStream_t s) {
    switch (t.P) {
#define FMM_CASE(Q) \
    case Q: launch_up<Q>(t, B, s); break;
        FMM_FOR_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
}

void dispatch_down(Tree& t, const Bufs& B, cudaStream_t s, bool log_kernel) {
    switch (t.P) {
#define FMM_CASE(Q)                                   \
    case Q:                                           \
        if (log_kernel) launch_down<Q, true>(t, B, s); \
        else launch_down<Q, false>(t, B, s);           \
        break;
        FMM_FOR_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
}

void dispatch_far(Tree& t, const Bufs& B, cudaStream_t s, bool log_kernel) {
    dispatch_up(t, B, s);
    dispatch_down(t, B, s, log_kernel);
}

// The deepest level's locals, which the FP32 evaluation does not form (its L2P
// uses the parents' locals): the L2L of that level for strength set 0, for the
// export of the local expansions only.
template <int P>
static void launch_folded_locals(Tree& t, const Bufs& B, cudaStream_t s) {
    const LevelList& L = t.level_boxes[t.Lmax - 1];
    if (L.count <= kWarpShiftMax)
        k_l2l_warp<P, float2, false><<<nblk(32 * (int64_t)L.count, 128), 128, 0, s>>>(
            L.d_ids, L.count, t.d_parent, t.d_child0, t.d_rho, t.d_center, t.d_box_m2l,
            static_cast<const float2*>(B.Lm2l), B.L64, nullptr, 0, t.p, t.PS);
    else
        k_l2l<P, float2, false><<<nblk(L.count, 128), 128, 0, s>>>(
            L.d_ids, L.count, t.d_parent, t.d_child0, t.d_rho, t.d_center, t.d_box_m2l,
            static_cast<const float2*>(B.Lm2l), B.L64, nullptr, 0, t.p, t.PS);
}

fmm_status complete_folded_locals(Tree& t, cudaStream_t s) {
    if (!fold_leaf_l2l(t)) return FMM_OK;
    const Bufs B = bufs(t, 0);
    switch (t.P) {
#define FMM_CASE(Q) \
    case Q: launch_folded_locals<Q>(t, B, s); break;
        FMM_FOR_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

static void dispatch_l2p(Tree& t, const Bufs& B, void* d_phi, cudaStream_t s) {
    switch (t.P) {
#define FMM_CASE(Q) \
    case Q: launch_l2p<Q>(t, B, d_phi, s); break;
        FMM_FOR_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
}

static void dispatch_l2p_log(Tree& t, const Bufs& B0, const Bufs& B1, void* d_phi, cudaStream_t s) {
    switch (t.P) {
#define FMM_CASE(Q) \
    case Q: launch_l2p_log<Q>(t, B0, B1, d_phi, s); break;
        FMM_FOR_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
}

// ------------------------------------------------------------- workspace

template <typename T>
static fmm_status ralloc(T** p, size_t bytes) {
    if (*p) cudaFree((void*)*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(bytes, 16));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error("device allocation failed (evaluation workspace)");
        return FMM_ERR_OOM;
    }
    FMM_CUDA(e);
    return FMM_OK;
}

// Evaluation workspace: `sets` strength sets (1 forward, 2 adjoint and
// logarithmic kernel).  The part that follows the tree shape and the
// expansion order (strengths, expansions, near field, slot-layout strengths)
// and the part that follows the work-item capacities of the coupling lists
// (partial sums of split boxes) are allocated separately, so that an
// evaluation can start on the tree before its lists exist.  Each is a no-op
// when nothing grew.
fmm_status alloc_eval_core(Tree& t, int sets) {
    if (t.eval_nbox == (size_t)t.nbox && t.eval_n == (size_t)t.n && t.eval_PS == t.PS && t.eval_path == t.path &&
        t.eval_sets >= sets && t.eval_slots == t.slot_alloc)
        return FMM_OK;
    sets = std::max(sets, t.eval_sets);
    ++t.eval_gen;
    const size_t nb = (size_t)t.nbox, n = (size_t)t.n, PS = (size_t)t.PS;
    const size_t cs = t.path == FMM_PATH_FP32 ? sizeof(float2) : sizeof(double2);
    fmm_status st;
    if ((st = ralloc(&t.d_gam, n * cs * sets))) return st;
    if ((st = ralloc(&t.d_near, n * sizeof(double2) * 3))) return st;
    if ((st = ralloc(&t.d_M64, nb * PS * sizeof(double2) * sets))) return st;
    if ((st = ralloc(&t.d_L64, nb * PS * sizeof(double2) * sets))) return st;
    if ((st = ralloc(&t.d_Lm2l, nb * PS * cs * sets))) return st;
    if ((st = ralloc(&t.d_M32, nb * PS * sizeof(float2) * sets))) return st;
    if ((st = ralloc(&t.d_L32, nb * PS * sizeof(float2) * sets))) return st;
    if (t.path == FMM_PATH_FP32 && m2l_tc_enabled() && (st = m2l_tc_prepare(t.P))) return st;
    // strengths in the slot layout: padding slots keep strength zero
    if ((st = ralloc(&t.d_gamp, (size_t)t.slot_alloc * cs))) return st;
    FMM_CUDA(cudaMemset(t.d_gamp, 0, (size_t)t.slot_alloc * cs));
    t.eval_slots = t.slot_alloc;
    // root locals are never written by the passes: they stay zero
    FMM_CUDA(cudaMemset(t.d_L64, 0, nb * PS * sizeof(double2) * sets));
    FMM_CUDA(cudaMemset(t.d_L32, 0, nb * PS * sizeof(float2) * sets));
    t.eval_nbox = nb;
    t.eval_n = n;
    t.eval_PS = t.PS;
    t.eval_path = t.path;
    t.eval_sets = sets;
    t.parts_stale = true;  // the partial sums follow the new set count / stride
    return FMM_OK;
}

fmm_status alloc_eval_parts(Tree& t) {
    if (!t.parts_stale && t.part_p2p_cap >= t.p2p_cap && t.part_m2l_cap >= t.m2l_cap && t.eval_ts >= t.max_leaf)
        return FMM_OK;
    ++t.eval_gen;
    const size_t PS = (size_t)t.PS;
    const size_t cs = t.path == FMM_PATH_FP32 ? sizeof(float2) : sizeof(double2);
    fmm_status st;
    if ((st = ralloc(&t.d_p2p_part, (size_t)t.p2p_cap * t.max_leaf * sizeof(double2) * 3))) return st;
    if ((st = ralloc(&t.d_m2l_part, (size_t)t.m2l_cap * PS * cs * t.eval_sets))) return st;
    t.part_p2p_cap = t.p2p_cap;
    t.part_m2l_cap = t.m2l_cap;
    t.eval_ts = t.max_leaf;
    t.parts_stale = false;
    return FMM_OK;
}

fmm_status alloc_eval(Tree& t, int sets) {
    fmm_status st = alloc_eval_core(t, sets);
    if (st) return st;
    return alloc_eval_parts(t);
}

// Strengths of one evaluation into sorted order and into the leaf slot layout.
void launch_gather(Tree& t, const Bufs& B, const double* d_gamma, cudaStream_t s) {
    const int n = (int)t.n;
    const double2* gin = reinterpret_cast<const double2*>(d_gamma);
    if (t.path == FMM_PATH_FP32) {
        // word 1 of the status area: set by the gather when a strength has a nonzero imaginary part
        // (the FP32 P2P then takes the complex form, else the real one)
        cudaMemsetAsync(t.d_status + 1, 0, sizeof(unsigned), s);
        k_gather32<<<nblk(n, 256), 256, 0, s>>>(gin, t.d_perm, t.d_slot_of, n, static_cast<float2*>(B.gam),
                                                static_cast<float*>(t.d_gamp), t.d_status + 1);
    }
    else
        k_gather64<<<nblk(n, 256), 256, 0, s>>>(gin, t.d_perm, t.d_slot_of, n, static_cast<double2*>(B.gam),
                                                static_cast<double2*>(t.d_gamp));
}

void launch_near(Tree& t, const Bufs& B, cudaStream_t s) { launch_p2p<false>(t, B, s); }
void launch_l2p_near(Tree& t, const Bufs& B, void* d_phi, cudaStream_t s) { dispatch_l2p(t, B, d_phi, s); }

// ---- persistent evaluation: stage table and launch ---------------------------
// The stage table follows the tree shape, the expansion order and the launch
// grids of the work items (the kernel reads the exact item counts on the
// device); it is rebuilt on the host for every evaluation and uploaded only
// when it changed (outside any stream capture: prepare_persistent runs before
// the evaluation is launched or captured).
static std::vector<PStage> persistent_stages(const Tree& t) {
    std::vector<PStage> far;
    auto add = [&](std::vector<PStage>& v, int type, long long nvb, const int32_t* ids, int cnt, int arg) {
        if (nvb <= 0) return;
        PStage g{};
        g.type = type;
        g.nvb = (int)nvb;
        g.ids = ids;
        g.cnt = cnt;
        g.arg = arg;
        v.push_back(g);
    };
    auto vb = [](long long threads) { return (threads + 127) / 128; };
    add(far, PT_GATHER, vb(t.n), nullptr, 0, 0);
    add(far, PT_P2M_T, vb(t.nleaf), t.leaves.d_ids, (int)t.nleaf, 0);
    for (int l = t.Lmax - 2; l >= 0; --l) {
        const LevelList& L = t.level_parents[l];
        if (!L.count) continue;
        const int how = p2m_parent_mode(t, l);
        if (how == 1) add(far, PT_P2M_T, vb(L.count), L.d_ids, L.count, 1);
        else if (how == 2) add(far, PT_P2M_W, vb(32LL * L.count), L.d_ids, L.count, 1);
    }
    const size_t n_p2m = far.size();  // stages that need the strengths only
    for (int l = t.Lmax - 2; l >= 0; --l) {
        const LevelList& L = t.level_parents[l];
        if (!L.count || p2m_parent_mode(t, l) != 0) continue;
        if (4LL * L.count <= kWarpShiftMax) add(far, PT_M2M_W, L.count, L.d_ids, L.count, 0);
        else add(far, PT_M2M_T, vb(4LL * L.count), L.d_ids, L.count, 0);
    }
    add(far, PT_M2L, vb(m2l_grid_items(t)), nullptr, 0, 0);
    add(far, PT_REDUCE, vb(32LL * t.nbox), nullptr, 0, 0);
    const bool fold = fold_leaf_l2l(t);
    const int lend = fold ? t.Lmax - 2 : t.Lmax - 1;
    for (int l = 0; l + 1 <= lend; ++l) {
        const LevelList& L = t.level_boxes[l + 1];
        if (!L.count) continue;
        const int all32 = fold && l + 1 == lend;
        if (L.count <= kWarpShiftMax) add(far, PT_L2L_W, vb(32LL * L.count), L.d_ids, L.count, all32);
        else add(far, PT_L2L_T, vb(L.count), L.d_ids, L.count, all32);
    }
    // dependencies: P2M stages wait for the gather, every later far-field stage for all far units before it
    long long before = 0;
    const long long gather_units = far[0].nvb;
    for (size_t i = 0; i < far.size(); ++i) {
        far[i].need_far = (i == 0) ? 0 : (i < n_p2m ? gather_units : before);
        far[i].need_p2p = 0;
        before += far[i].nvb;
    }
    // P2P (4 items per unit, one per warp) in chunks after every far-field stage from the leaves' P2M on
    const long long np2p = (p2p_grid_items(t) + 3) / 4;
    const int slots = std::max<int>(1, (int)far.size() - 1);
    std::vector<PStage> st;
    long long done_p2p = 0;
    for (size_t i = 0; i < far.size(); ++i) {
        st.push_back(far[i]);
        if (i == 0) continue;
        const long long upto = np2p * (long long)i / slots;
        if (upto > done_p2p) {
            PStage g{};
            g.type = PT_P2P;
            g.nvb = (int)(upto - done_p2p);
            g.vb0 = (int)done_p2p;
            g.need_far = gather_units;
            st.push_back(g);
            done_p2p = upto;
        }
    }
    PStage l2p{};
    l2p.type = PT_L2P;
    l2p.nvb = (int)((t.n + 127) / 128);
    l2p.need_far = before;
    l2p.need_p2p = np2p;
    st.push_back(l2p);
    long long tk = 0;
    for (auto& g : st) {
        g.ticket0 = tk;
        tk += g.nvb;
    }
    return st;
}

fmm_status prepare_persistent(Tree& t) {
    if (t.path != FMM_PATH_FP32) {
        set_error("FMM_FLAG_PERSISTENT: the persistent evaluation runs the FP32 path only");
        return FMM_ERR_INVALID_ARG;
    }
    const std::vector<PStage> st = persistent_stages(t);
    if ((int)st.size() > kMaxPStages) {
        set_error("FMM_FLAG_PERSISTENT: too many stages for the work queue");
        return FMM_ERR_INVALID_ARG;
    }
    const size_t bytes = st.size() * sizeof(PStage);
    if (t.d_pstage && t.h_pstage.size() == bytes && memcmp(t.h_pstage.data(), st.data(), bytes) == 0) return FMM_OK;
    if (!t.d_pstage) {
        FMM_CUDA(cudaMalloc(&t.d_pstage, kMaxPStages * sizeof(PStage)));
        FMM_CUDA(cudaMalloc((void**)&t.d_pers, 4 * sizeof(unsigned long long)));
    }
    FMM_CUDA(cudaMemcpy(t.d_pstage, st.data(), bytes, cudaMemcpyHostToDevice));
    t.h_pstage.assign(reinterpret_cast<const char*>(st.data()), reinterpret_cast<const char*>(st.data()) + bytes);
    t.npstage = (int)st.size();
    t.pstage_total = st.back().ticket0 + st.back().nvb;
    return FMM_OK;
}

template <int P>
static fmm_status launch_persistent(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s) {
    static int occ = 0;
    if (!occ) {
        FMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval_persistent<P>, 128, 0));
        occ = std::max(occ, 1);
    }
    const Bufs B = bufs(t, 0);
    const P2PLayout pl = p2p_pair_layout(t.max_leaf);
    PArgs a{};
    a.st = static_cast<const PStage*>(t.d_pstage);
    a.nst = t.npstage;
    a.total = t.pstage_total;
    a.ctr = t.d_pers;
    a.status = t.d_status;
    a.cplx = t.d_status + 1;
    a.wait_ns = 4000000000ull;  // 4 s of the global timer: far beyond any stage
    a.n = (int)t.n;
    a.nbox = (int)t.nbox;
    a.p = t.p;
    a.PS = t.PS;
    a.lay = pl.tpl * 100 + pl.lt;
    a.pad = (int)(t.nleaf * t.leaf_cap);
    a.TS = t.max_leaf;
    a.gin = reinterpret_cast<const double2*>(d_gamma);
    a.perm = t.d_perm;
    a.slot_of = t.d_slot_of;
    a.bstart = t.d_bstart;
    a.bcount = t.d_bcount;
    a.child0 = t.d_child0;
    a.parent = t.d_parent;
    a.leaf_of = t.d_leaf_of;
    a.fold_par = t.d_fold_par;
    a.pslot = t.d_pslot;
    a.soff = t.d_soff;
    a.woff = t.d_woff;
    a.widx = t.d_widx;
    a.m2l_rows = t.d_m2l_rows;
    a.chl = t.d_chl;
    a.pos4 = t.d_pos4;
    a.rho32 = t.d_rho32;
    a.rho = t.d_rho;
    a.center = t.d_center;
    a.box_m2l = t.d_box_m2l;
    a.srng = t.d_srng;
    a.leaf_items = t.d_leaf_items;
    a.m2l_items = t.d_m2l_items;
    a.p2p_items = t.d_p2p_items;
    a.n_m2l = item_count(t, 3);
    a.n_p2p = item_count(t, 2);
    a.p2p_nheavy = t.d_m2l_rowctr + kM2LItemPairsMax + 1;
    a.p2p_rows = t.d_p2p_rows;
    a.p2p_cap = t.p2p_cap;
    a.tfirst = t.n_src > 0 ? t.d_nsrc : nullptr;
    a.near_slot = t.n_src > 0 ? t.d_slot_of : nullptr;
    a.posq = static_cast<const ulonglong2*>(t.d_posp);
    a.gam = static_cast<float2*>(B.gam);
    a.gamp = static_cast<float*>(t.d_gamp);
    a.M32 = B.M32;
    a.M64 = B.M64;
    a.Lm2l = static_cast<float2*>(B.Lm2l);
    a.m2l_part = static_cast<float2*>(B.m2l_part);
    a.L64 = B.L64;
    a.L32 = B.L32;
    a.nearv = static_cast<float2*>(B.near);
    a.p2p_part = static_cast<float2*>(B.p2p_part);
    a.out = static_cast<float2*>(d_phi);
    FMM_CUDA(cudaMemsetAsync(t.d_pers, 0, 4 * sizeof(unsigned long long), s));
    FMM_CUDA(cudaMemsetAsync(t.d_status + 1, 0, sizeof(unsigned), s));  // the complex-strength flag
    const long long grid = std::min<long long>((long long)occ * t.num_sms, std::max<long long>(t.pstage_total, 1));
    k_eval_persistent<P><<<(int)grid, 128, 0, s>>>(a);
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

fmm_status run_eval_persistent(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s) {
    t.p2p_funcs.clear();
    t.timing_valid = false;
    switch (t.P) {
#define FMM_CASE(Q) \
    case Q: return launch_persistent<Q>(t, d_gamma, d_phi, s);
        FMM_FOR_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
    set_error("unsupported expansion order");
    return FMM_ERR_INVALID_ARG;
}

// One evaluation: gather strengths into sorted order, then fork P2P onto the
// auxiliary stream while the far field (P2M, M2M, M2L, L2L) runs on the
// caller's stream, join, and finish with L2P + near + unpermute.
fmm_status run_eval(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s) {
    t.p2p_funcs.clear();
    const bool timing = t.flags & FMM_FLAG_TIMING;
    const bool serial = t.flags & FMM_FLAG_SERIAL;
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[0], s));
    const Bufs B = bufs(t, 0);
    launch_gather(t, B, d_gamma, s);
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[1], s));
    if (!serial) {
        FMM_CUDA(cudaEventRecord(t.ev_fork, s));
        FMM_CUDA(cudaStreamWaitEvent(t.s_far, t.ev_fork, 0));
        FMM_CUDA(cudaStreamWaitEvent(t.s_aux, t.ev_fork, 0));
        dispatch_far(t, B, t.s_far);
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[4], t.s_far));
        FMM_CUDA(cudaEventRecord(t.ev_join_far, t.s_far));
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[5], t.s_aux));
        launch_p2p<false>(t, B, t.s_aux);
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[6], t.s_aux));
        FMM_CUDA(cudaEventRecord(t.ev_join, t.s_aux));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join_far, 0));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
    } else {
        dispatch_far(t, B, s);
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[4], s));
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[5], s));
        launch_p2p<false>(t, B, s);
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[6], s));
    }
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[8], s));  // both halves done: L2P + combine from here
    dispatch_l2p(t, B, d_phi, s);
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[7], s));
    FMM_CUDA(cudaGetLastError());
    t.timing_valid = timing;
    return FMM_OK;
}

// Logarithmic kernel (Sec. 3.3): the two real-strength sets' far fields on two
// high-priority streams (their latency-bound kernels overlap), the
// complex-strength P2P on the low-priority stream, then one L2P for both.
// Needs a workspace of two strength sets.
fmm_status run_eval_log(Tree& t, const double* d_gamma, void* d_phi, cudaStream_t s) {
    const int n = (int)t.n;
    t.p2p_funcs.clear();
    const bool timing = t.flags & FMM_FLAG_TIMING;
    const bool serial = t.flags & FMM_FLAG_SERIAL;
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[0], s));
    const double2* gin = reinterpret_cast<const double2*>(d_gamma);
    const Bufs B0 = bufs(t, 0), B1 = bufs(t, 1);
    if (t.path == FMM_PATH_FP32)
        k_gather_log32<<<nblk(n, 256), 256, 0, s>>>(gin, t.d_perm, t.d_slot_of, n, static_cast<float2*>(B0.gam),
                                                    static_cast<float2*>(B1.gam), static_cast<float*>(t.d_gamp));
    else
        k_gather_log64<<<nblk(n, 256), 256, 0, s>>>(gin, t.d_perm, t.d_slot_of, n, static_cast<double2*>(B0.gam),
                                                    static_cast<double2*>(B1.gam), static_cast<double2*>(t.d_gamp));
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[1], s));
    cudaStream_t sf = serial ? s : t.s_far, sf2 = serial ? s : t.s_far2, sa = serial ? s : t.s_aux;
    if (!serial) {
        FMM_CUDA(cudaEventRecord(t.ev_fork, s));
        FMM_CUDA(cudaStreamWaitEvent(t.s_far, t.ev_fork, 0));
        FMM_CUDA(cudaStreamWaitEvent(t.s_far2, t.ev_fork, 0));
        FMM_CUDA(cudaStreamWaitEvent(t.s_aux, t.ev_fork, 0));
    }
    {
        // phase events cover set 0 only (set 1 runs beside it)
        dispatch_far(t, B0, sf, true);
        if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[4], sf));
        const int flags = t.flags;
        t.flags &= ~FMM_FLAG_TIMING;
        dispatch_far(t, B1, sf2, true);
        t.flags = flags;
    }
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[5], sa));
    launch_p2p<true>(t, B0, sa);
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[6], sa));
    if (!serial) {
        FMM_CUDA(cudaEventRecord(t.ev_join_far, t.s_far));
        FMM_CUDA(cudaEventRecord(t.ev_join_far2, t.s_far2));
        FMM_CUDA(cudaEventRecord(t.ev_join, t.s_aux));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join_far, 0));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join_far2, 0));
        FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
    }
    dispatch_l2p_log(t, B0, B1, d_phi, s);
    if (timing) FMM_CUDA(cudaEventRecord(t.ev_t[7], s));
    FMM_CUDA(cudaGetLastError());
    t.timing_valid = timing;
    return FMM_OK;
}

}  // namespace fmm
