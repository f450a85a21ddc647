// M2L of the FP32 path on the 5th-generation tensor cores (tcgen05).
//
// The multipole-to-local translation (Sec. 2.1, the M2L step of Fig 2.2) in
// the scaled form used by every pass,
//     bt_l += g_l * w_l,   w_l = sum_k C(k+l, l) v_k,
//     v_k = (rho_M u)^k at_k,   g_l = u (-rho_L u)^l,   u = 1/(c_L - c_M),
// is a FIXED real matrix B[l][k] = C(k+l, l) (a Hankel matrix of binomial
// coefficients) applied to a power-scaled coefficient vector v, with
// pair-dependent diagonal scalings on both sides.  Only the constant product
// w = B v is a dense contraction; it runs on the tensor cores, the two diagonal
// scalings and the sum over the weak list stay on the CUDA cores.
//
// Work layout: a CTA takes 128 consecutive rows of the M2L row order, one
// work item (a target box and up to 192 entries of its weak list) per thread.
// The row order puts every full item first and then the boxes' shorter last
// items by decreasing length, so the threads of a CTA, which step through
// their pairs in lockstep, have about the same number of pairs.  Step j treats the j-th
// weak entry of every item at once: each thread writes its v (real and
// imaginary parts, TF32 hi/lo split) as row `thread` of the A operands, which
// live in tensor memory (tcgen05.st, lane = thread); one elected thread issues
// the MMAs (M = 128 rows, N = l, K = k; B from shared memory) into a TMEM
// accumulator, and each thread reads its own row back two steps later and
// adds g_l w_l to its register accumulator.  Two accumulator stages keep the
// MMAs of step j running while the threads prepare step j+1 and finish step
// j-1; the A operands are rewritten only after the previous step's MMAs have
// completed, a wait placed after the CUDA-core work of the step.
//
// The tensor-core block covers k < KT and l < NT (multiples of 8 and 16); when
// p exceeds them by one or two (p = 17: KT = NT = 16) the remaining row and
// column of B are applied on the CUDA cores with the coefficients as
// immediates, which keeps the operands small enough for three CTAs per SM.
//
// Logarithmic kernel (LOG): the same contraction, plus the constant term of
// the log local, b0 += Re(at_0) ln|c_L - c_M| - sum_{k>=1} Re(v_k)/k, summed on
// the CUDA cores from the v_k each thread forms anyway and written to slot P.
//
// Precision: 3xTF32.  v = v_hi + v_lo and B = B_hi + B_lo with TF32 parts, and
// w = v_lo B_hi + v_hi B_lo + v_hi B_hi accumulated in FP32 (the v_lo B_lo term
// is below FP32 rounding): about 2^-21 relative per product.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <utility>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr int kTcThreads = kM2LTcRows;  // = MMA rows M = items per CTA
constexpr int kTabN = 32;        // B table covers k, l < 32 (orders up to 32)

// ---- B = C(k+l, l) split into TF32 hi + lo, evaluated at compile time -------
// Binomials exactly in 64-bit integers (Pascal's rule; C(62,31) < 2^63), then
// rounded to 11 significant bits (TF32) with ties away from zero.
constexpr double tf32_round(double x) {
    if (x == 0.0) return 0.0;
    const double a = x < 0.0 ? -x : x;
    double s = 1.0;
    while (a >= 2048.0 * s) s *= 2.0;
    while (a < 1024.0 * s) s *= 0.5;
    const double r = static_cast<double>(static_cast<long long>(a / s + 0.5)) * s;
    return x < 0.0 ? -r : r;
}
struct TcTable {
    float hi[kTabN][kTabN];
    float lo[kTabN][kTabN];
    constexpr TcTable() : hi(), lo() {
        unsigned long long pas[2 * kTabN][2 * kTabN] = {};
        for (int n = 0; n < 2 * kTabN; ++n) {
            pas[n][0] = 1;
            for (int k = 1; k <= n; ++k) pas[n][k] = pas[n - 1][k - 1] + (k < n ? pas[n - 1][k] : 0);
        }
        for (int l = 0; l < kTabN; ++l)
            for (int k = 0; k < kTabN; ++k) {
                const double c = static_cast<double>(pas[k + l][l]);
                const double h = tf32_round(c);
                hi[l][k] = static_cast<float>(h);
                lo[l][k] = static_cast<float>(tf32_round(c - h));
            }
    }
};
__device__ const TcTable g_tc_table = TcTable();

// FP32 binomial as an immediate for the CUDA-core edge of B.
template <int N, int K>
struct Bc {
    static constexpr float v = static_cast<float>(binom_d(N, K));
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// x = hi + lo with hi rounded to TF32 (ties away from zero; finite x) and lo
// the exact remainder, which the tensor core reads truncated to TF32.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
    hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
    lo = x - hi;
}

// Shared-memory matrix descriptor of a K-major operand without swizzling.  The
// operand is stored as 8-row x 16-byte core matrices; lbo = byte distance of
// core matrices adjacent in K, sbo = adjacent in the row (M or N) dimension.
// Bits: [0,14) address>>4, [16,30) lbo>>4, [32,46) sbo>>4, [46,48) = 1
// (descriptor version), base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr >> 4) & 0x3fffu) | (static_cast<uint64_t>((lbo >> 4) & 0x3fffu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D f32 (bits 4-5 = 1), A and B tf32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N>>3 at bit 17,
// M>>4 at bit 24.
template <int N>
__host__ __device__ constexpr uint32_t idesc_tf32_m128() {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false when the phase did not complete within `limit` tries.
constexpr int kMbarTries = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit = kMbarTries) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&r)[8]) {
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 consecutive 32-bit TMEM columns of this thread's lane <- registers.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(r[0])), "r"(__float_as_uint(r[1])), "r"(__float_as_uint(r[2])),
                 "r"(__float_as_uint(r[3])), "r"(__float_as_uint(r[4])), "r"(__float_as_uint(r[5])),
                 "r"(__float_as_uint(r[6])), "r"(__float_as_uint(r[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ bool elect_one() {
    uint32_t pred;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "elect.sync _|P, 0xffffffff;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(pred));
    return pred != 0;
}

// MMA with A from tensor memory (lanes = rows, one TF32 per column) and B from
// shared memory.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Float offset of element (row r, column k) of a K-major no-swizzle operand
// with K columns: core matrix (r/8, k/4) at (r/8)*8K + (k/4)*32, row r%8 at
// 4*(r%8) inside it.
template <int K>
__host__ __device__ constexpr int op_off(int r, int k) {
    return (r >> 3) * (8 * K) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

template <int P>
struct TcShape {
    static constexpr int KT = (P % 8 <= 2) ? P / 8 * 8 : (P + 7) / 8 * 8;      // k on the tensor cores
    static constexpr int NT = (P % 16 <= 2) ? P / 16 * 16 : (P + 15) / 16 * 16;  // l on the tensor cores
    static constexpr int KTAIL = P > KT ? P - KT : 0;
    static constexpr int NTAIL = P > NT ? P - NT : 0;
    static constexpr int KW = KT < P ? KT : P;  // k columns holding data
    static constexpr int B_FLOATS = NT * KT;
    // TMEM columns: A operands [hi_re, lo_re, hi_im, lo_im] x KT, then 2 stages x (re, im) x NT
    static constexpr int COL_D = 4 * KT;
    static constexpr int COLS_USED = 4 * KT + 4 * NT;
    static constexpr int TCOLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                               : COLS_USED <= 256 ? 256 : 512;
    // B: [hi, lo] in shared memory; mbarrier; TMEM address
    static constexpr size_t SMEM = (size_t)(2 * B_FLOATS) * 4 + 8 + 8;
    static_assert(KT >= 8 && NT >= 16 && KTAIL <= 2 && NTAIL <= 2 && COLS_USED <= 256, "tensor-core M2L shape");
};

// Per-pair values carried from the step that prepares a pair to the step that
// reads its accumulator back.
template <int P>
struct PairState {
    float2 u, beta;
    float2 vt[TcShape<P>::KTAIL > 0 ? TcShape<P>::KTAIL : 1];  // v_k, k >= KT
    float2 wt[TcShape<P>::NTAIL > 0 ? TcShape<P>::NTAIL : 1];  // w_l, l >= NT (CUDA cores)
};

template <int KT, int NT, int... L>
__device__ __forceinline__ void ktail_row(float (&wr)[NT], float (&wi)[NT], const float2 v,
                                          std::integer_sequence<int, L...>) {
    ((wr[L] = fmaf(Bc<KT + L, L>::v, v.x, wr[L])), ...);
    ((wi[L] = fmaf(Bc<KT + L, L>::v, v.y, wi[L])), ...);
}
template <int P, int L, int... K>
__device__ __forceinline__ float2 ltail_col(const float2 (&v)[P], std::integer_sequence<int, K...>) {
    float2 w = make_float2(0.f, 0.f);
    ((w.x = fmaf(Bc<K + L, L>::v, v[K].x, w.x)), ...);
    ((w.y = fmaf(Bc<K + L, L>::v, v[K].y, w.y)), ...);
    return w;
}
template <int P, int NT, int NW, int... T>
__device__ __forceinline__ void ltail_all(const float2 (&v)[P], float2 (&wt)[NW], std::integer_sequence<int, T...>) {
    ((wt[T] = ltail_col<P, NT + T>(v, std::make_integer_sequence<int, P>{})), ...);
}

template <int P, bool LOG>
__global__ void __launch_bounds__(kTcThreads, P <= 18 ? 3 : 2)
    k_m2l_tc(const int4* __restrict__ items, const int32_t* __restrict__ rows,
             const unsigned long long* __restrict__ nitems, const int32_t* __restrict__ woff,
             const int32_t* __restrict__ widx, const float4* __restrict__ chl, const float* __restrict__ rho32,
             const float2* __restrict__ M32, float2* __restrict__ Lm2l, float2* __restrict__ part, int PS,
             unsigned* status) {
    using S = TcShape<P>;
    constexpr int KT = S::KT, NT = S::NT, KW = S::KW, B_FLOATS = S::B_FLOATS, COL_D = S::COL_D;
    constexpr int NA = (P + 1) / 2;  // float4 loads of one multipole (PS even)
    extern __shared__ __align__(1024) float sm[];
    float* sB = sm;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 2 * B_FLOATS);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
    __shared__ int s_len[kTcThreads / 32];

    const int nit = static_cast<int>(*nitems);
    if (blockIdx.x * kTcThreads >= nit) return;  // CTA-uniform
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = blockIdx.x * kTcThreads + tid;
    const bool has = row < nit;
    int it = 0;  // work item of this row
    int4 item = make_int4(0, 0, 0, -1);
    if (has) {
        it = rows[row];
        item = items[it];
    }
    const int len = has ? item.z - item.y : 0;

    // B operand (k < KT, l < NT; zero past p), K-major in shared memory
    for (int e = tid; e < B_FLOATS; e += kTcThreads) {
        const int l = e / KT, k = e % KT;
        const bool in = l < P && k < P;
        sB[op_off<KT>(l, k)] = in ? g_tc_table.hi[l][k] : 0.f;
        sB[B_FLOATS + op_off<KT>(l, k)] = in ? g_tc_table.lo[l][k] : 0.f;
    }
    {
        int m = len;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0) s_len[warp] = m;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(static_cast<uint32_t>(S::TCOLS))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();  // B, written by the threads, is read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    int J = 0;
#pragma unroll
    for (int w = 0; w < kTcThreads / 32; ++w) J = max(J, s_len[w]);

    const int b = item.x;
    float4 ct = make_float4(0.f, 0.f, 0.f, 0.f);
    float rt = 0.f;
    const int32_t* wl = widx;
    if (has) {
        ct = chl[b];
        rt = rho32[b];
        wl = widx + woff[b] + item.y;
    }
    float2 acc[P];
#pragma unroll
    for (int l = 0; l < P; ++l) acc[l] = make_float2(0.f, 0.f);
    float b0 = 0.f;  // log kernel: constant term

    // inputs of the next pair (loaded one step ahead) and the index after it
    float4 ncs = make_float4(1.f, 1.f, 0.f, 0.f), naa[NA];
    float nrs = 0.f;
#pragma unroll
    for (int q = 0; q < NA; ++q) naa[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int s_next = 0;
    auto fetch = [&](int s) {
        ncs = chl[s];
        nrs = rho32[s];
        const float4* src = reinterpret_cast<const float4*>(M32 + (size_t)s * PS);
#pragma unroll
        for (int q = 0; q < NA; ++q) naa[q] = src[q];
    };
    if (len > 0) fetch(wl[0]);
    if (len > 1) s_next = wl[1];

    PairState<P> g1{}, g2{};  // pairs j-1 and j-2
    bool timed_out = false, stopped = false;
    const uint32_t trow = tbase + (static_cast<uint32_t>(warp * 32) << 16);  // this thread's TMEM lane
    const uint64_t bdesc0 = smem_desc(smem_u32(sB), 128, 8 * KT * 4);
    for (int j = 0; j <= J + 1; ++j) {
        const int st = j & 1;
        PairState<P> cur{};
        if (j < J) {
            // (b) pair j: v_k = alpha^k at_k (rows without a pair this step compute
            // throwaway values: an MMA row depends only on its own A row)
            const float dx = (ct.x - ncs.x) + (ct.z - ncs.z);
            const float dy = (ct.y - ncs.y) + (ct.w - ncs.w);
            const float r2 = fmaf(dx, dx, dy * dy);
            const float inv = rcp_approx(r2);  // hardware reciprocal (within about one ulp)
            cur.u = make_float2(dx * inv, -dy * inv);  // 1/d, d = c_target - c_source
            const float2 alpha = make_float2(nrs * cur.u.x, nrs * cur.u.y);
            cur.beta = make_float2(-rt * cur.u.x, -rt * cur.u.y);
            float2 v[P];
            float2 ap = make_float2(1.f, 0.f);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float4 q = naa[k / 2];
                const float2 a = (k & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
                v[k] = cmul(ap, a);
                if (k + 1 < P) ap = cmul(ap, alpha);
            }
            if constexpr (LOG) {
                if (j < len) {
                    float ls = 0.f;
#pragma unroll
                    for (int k = 1; k < P; ++k) ls = fmaf(-1.0f / k, v[k].x, ls);
                    b0 += fmaf(0.5f * logf(r2), naa[0].x, ls);
                }
            }
            if constexpr (S::KTAIL > 0) {
#pragma unroll
                for (int k = 0; k < S::KTAIL; ++k) cur.vt[k] = v[KT + k];
            }
            if constexpr (S::NTAIL > 0)
                ltail_all<P, NT, S::NTAIL>(v, cur.wt, std::make_integer_sequence<int, S::NTAIL>{});
            if (j + 1 < len) {
                fetch(s_next);
                if (j + 2 < len) s_next = wl[j + 2];
            }
            // the MMAs of pair j-1 read the A operands: wait for them, then store pair j
            if (j >= 1) {
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(mbar), static_cast<uint32_t>((j - 1) & 1))))
                    timed_out = true;
                tc_fence_after();
            }
            if (!timed_out) {
#pragma unroll
                for (int c8 = 0; c8 < KT / 8; ++c8) {
                    float hr[8], lr[8], hi[8], li[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int k = 8 * c8 + e;
                        const float2 x = k < KW ? v[k < KW ? k : 0] : make_float2(0.f, 0.f);
                        tf32_split(x.x, hr[e], lr[e]);
                        tf32_split(x.y, hi[e], li[e]);
                    }
                    tmem_st8(trow + 0 * KT + 8 * c8, hr);
                    tmem_st8(trow + 1 * KT + 8 * c8, lr);
                    tmem_st8(trow + 2 * KT + 8 * c8, hi);
                    tmem_st8(trow + 3 * KT + 8 * c8, li);
                }
                tmem_wait_st();
            }
        } else if (j == J && J >= 1) {
            // no pair left: the last MMAs still have to finish before their accumulator is read
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(mbar), static_cast<uint32_t>((j - 1) & 1))))
                timed_out = true;
            tc_fence_after();
        }
        // (c) pair j-2: w = TMEM row (+ the CUDA-core edge of B), acc += g_l w_l
        if (j >= 2 && !timed_out) {
            float wr[NT], wi[NT];
            const uint32_t col = trow + COL_D + st * 2 * NT;
#pragma unroll
            for (int q = 0; q < NT / 8; ++q) {
                float r8[8], i8[8];
                tmem_ld8(col + 8 * q, r8);
                tmem_ld8(col + NT + 8 * q, i8);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    wr[8 * q + e] = r8[e];
                    wi[8 * q + e] = i8[e];
                }
            }
            tmem_wait_ld();
#pragma unroll
            for (int l = 0; l < NT; ++l) asm volatile("" : "+f"(wr[l]), "+f"(wi[l]));
            if (j - 2 < len) {
                if constexpr (S::KTAIL > 0) ktail_row<KT, NT>(wr, wi, g2.vt[0], std::make_integer_sequence<int, NT>{});
                if constexpr (S::KTAIL > 1)
                    ktail_row<KT + 1, NT>(wr, wi, g2.vt[S::KTAIL > 1 ? 1 : 0], std::make_integer_sequence<int, NT>{});
                float2 g = g2.u;
#pragma unroll
                for (int l = 0; l < P; ++l) {
                    const float2 w = l < NT ? make_float2(wr[l < NT ? l : 0], wi[l < NT ? l : 0])
                                            : g2.wt[l >= NT ? l - NT : 0];
                    acc[l] = cfma(g, w, acc[l]);
                    g = cmul(g, g2.beta);
                }
            }
        }
        g2 = g1;
        g1 = cur;
        // (d) MMAs of pair j into accumulator stage st
        tc_fence_before();
        if (__syncthreads_or(timed_out ? 1 : 0)) {
            stopped = true;
            break;
        }
        if (warp == 0 && j < J) {
            tc_fence_after();
            if (elect_one()) {
                constexpr uint32_t ID = idesc_tf32_m128<NT>();
                constexpr uint64_t BLO = (B_FLOATS * 4) >> 4;  // descriptor address step to B_lo
#pragma unroll
                for (int c = 0; c < 2; ++c) {  // real, imaginary part
                    const uint32_t d = tbase + static_cast<uint32_t>(COL_D + st * 2 * NT + c * NT);
                    const uint32_t ahi = tbase + static_cast<uint32_t>(2 * c * KT), alo = ahi + KT;
                    const uint32_t as[3] = {alo, ahi, ahi};
                    const uint64_t bs[3] = {bdesc0, bdesc0 + BLO, bdesc0};
#pragma unroll
                    for (int pass = 0; pass < 3; ++pass) {
#pragma unroll
                        for (int s = 0; s < KT / 8; ++s)  // 8 k per MMA: 8 TMEM columns of A, 256 bytes of B
                            mma_tf32_ts(d, as[pass] + 8 * s, bs[pass] + (256 >> 4) * s, ID, (pass | s) ? 1u : 0u);
                    }
                }
                mma_commit(smem_u32(mbar));
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    stopped = __syncthreads_or((stopped || timed_out) ? 1 : 0) != 0;
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(static_cast<uint32_t>(S::TCOLS))
                     : "memory");
    }
    if (stopped) {
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
        return;
    }
    // a box with one item: its M2L sum; otherwise the item's partial sum, which
    // k_reduce_m2l adds up in item order
    if (!has) return;
    float2* out = item.w < 0 ? Lm2l + (size_t)b * PS : part + (size_t)it * PS;
#pragma unroll
    for (int l = 0; l < P; ++l) out[l] = acc[l];
    if constexpr (LOG) out[P] = make_float2(b0, 0.f);
}

template <int P, bool LOG>
void launch_tc(const Tree& t, const float2* M32, float2* Lm2l, float2* part, cudaStream_t s) {
    const int grid = static_cast<int>(std::max<long long>((m2l_grid_items(t) + kTcThreads - 1) / kTcThreads, 1));
    k_m2l_tc<P, LOG><<<grid, kTcThreads, TcShape<P>::SMEM, s>>>(
        t.d_m2l_items, t.d_m2l_rows, reinterpret_cast<const unsigned long long*>(t.d_status) + 4, t.d_woff, t.d_widx,
        t.d_chl, t.d_rho32, M32, Lm2l, part, t.PS, t.d_status);
}

template <int P>
cudaError_t prepare_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(TcShape<P>::SMEM));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_m2l_tc<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TcShape<P>::SMEM));
}

// Self-test of the bounded mbarrier wait: a barrier nothing arrives at; the
// wait must give up after `limit` tries and report ST_TIMEOUT.
__global__ void k_selftest_mbar(int limit, unsigned* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0u, limit)) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

void launch_selftest_mbar(int limit, unsigned* status, cudaStream_t s) {
    k_selftest_mbar<<<1, 32, 0, s>>>(limit, status);
}

bool m2l_tc_enabled() {
    static const bool on = [] {
        const char* e = getenv("FMM_M2L_TC");
        return !(e && e[0] == '0');
    }();
    return on;
}

#define FMM_TC_ORDERS(X) X(4) X(8) X(12) X(16) X(17) X(20) X(24) X(28) X(32)

fmm_status m2l_tc_prepare(int P) {
    cudaError_t e = cudaSuccess;
    switch (P) {
#define FMM_CASE(Q) \
    case Q: e = prepare_tc<Q>(); break;
        FMM_TC_ORDERS(FMM_CASE)
#undef FMM_CASE
        default: break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_m2l_tc)");
    return FMM_OK;
}

void launch_m2l_tc(const Tree& t, const float2* M32, float2* Lm2l, float2* part, bool log_kernel,
                   cudaStream_t s) {
    switch (t.P) {
#define FMM_CASE(Q)                                            \
    case Q:                                                    \
        if (log_kernel) launch_tc<Q, true>(t, M32, Lm2l, part, s); \
        else launch_tc<Q, false>(t, M32, Lm2l, part, s);           \
        break;
        FMM_TC_ORDERS(FMM_CASE)
#undef FMM_CASE
        default: break;
    }
}
#undef FMM_TC_ORDERS

}  // namespace fmm
