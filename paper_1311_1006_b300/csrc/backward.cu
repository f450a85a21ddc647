// Adjoint of the FMM evaluation with the tree frozen.
//
// For the real loss L = sum_i w_i Re Phi_i + v_i Im Phi_i (upstream gphi = w + i v)
// put c = conj(gphi).  Then L = Re sum_i c_i Phi_i and, by the chain rule on the
// holomorphic kernel Gamma_j / (z_i - z_j):
//   dL/dRe Gamma_k + i dL/dIm Gamma_k = -conj(Psi_k),   Psi(z) = sum_i c_i / (z - z_i)
//   dL/dx_k = Re D_k,  dL/dy_k = -Im D_k,   D_k = c_k Phi'(z_k) - Gamma_k Psi'(z_k)
// with Phi'(z) = -sum_j Gamma_j/(z - z_j)^2 and Psi' likewise (pairs with
// z_j == z_k excluded, as in the forward sum).  Psi is a second FMM over the
// same tree with strengths c; Psi' and Phi' are the derivatives of the two
// local expansions (far part) plus a fused near-field sum of u and u^2,
// u = 1/(z_k - z_j).  So one adjoint = the far field of two strength sets
// + one P2P pass with three outputs + one L2P pass that assembles both
// gradients in the caller's order.
#include <cuda_runtime.h>

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

static inline int nblk(int64_t n, int b) { return (int)std::max<int64_t>((n + b - 1) / b, 1); }

constexpr int kBWarps = 8;
constexpr int kBChunk32 = 128;
constexpr int kBChunk64 = 96;

// sorted strengths of both sets: set 0 = Gamma, set 1 = c = conj(gphi); on the
// FP32 path also both sets in the leaf slot layout of the packed P2P (slot
// pairs interleaved as (re[2m], re[2m+1], im[2m], im[2m+1]))
template <typename C>
__global__ void k_gather_bwd(const double2* __restrict__ gam, const double2* __restrict__ gphi,
                             const int32_t* __restrict__ perm, const int32_t* __restrict__ slot_of, int n, C* s0,
                             C* s1, float* p0, float* p1) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = perm[i];
    const double2 a = gam[j], g = gphi[j];
    s0[i].x = a.x;
    s0[i].y = a.y;
    s1[i].x = g.x;
    s1[i].y = -g.y;
    if (p0 != nullptr) {
        const int slot = slot_of[i];
        float* f0 = p0 + 4 * (slot >> 1) + (slot & 1);
        float* f1 = p1 + 4 * (slot >> 1) + (slot & 1);
        f0[0] = (float)a.x;
        f0[2] = (float)a.y;
        f1[0] = (float)g.x;
        f1[2] = (float)-g.y;
    }
}

// ---- FP32 adjoint near field with packed f32x2 arithmetic --------------------
// The forward P2P's work items, slot layout and lane layout (k_p2p_pairs): a
// lane takes a pair of source slots per step and one target, every instruction
// a 2-wide FP32 operation; per pair three sums with u = 1/(z_t - z_s):
//     Psi += c_s u,   Psi' += -c_s u^2,   Phi' += -Gamma_s u^2,
// from the hi/lo coordinates (close pairs keep full FP32 relative accuracy).
// Coincident pairs give d = 0 and add 0 (|d|^2 carries a 1e-37 guard); padding
// slots have zero strengths.
struct BwdSrcPair {
    f2x x, y, xl, yl, cr, ci, ncr, nci, gr, ngr, ngi;
};
__device__ __forceinline__ BwdSrcPair bwd_src_pair(const ulonglong2 a, const ulonglong2 b, const ulonglong2 g,
                                                   const ulonglong2 c) {
    const f2x m1 = f2pk(-1.f, -1.f);
    BwdSrcPair s;
    s.x = a.x;
    s.y = a.y;
    s.xl = b.x;
    s.yl = b.y;
    s.cr = c.x;
    s.ci = c.y;
    s.ncr = f2mul(c.x, m1);
    s.nci = f2mul(c.y, m1);
    s.gr = g.x;
    s.ngr = f2mul(g.x, m1);
    s.ngi = f2mul(g.y, m1);
    return s;
}
struct BwdAcc {
    f2x pr, pi, qr, qi, fr, fi;  // Psi, Psi', Phi' (re, im); each holds the even- and odd-slot sums
};
__device__ __forceinline__ void bwd_pair(const f2x tx, const f2x ty, const f2x txl, const f2x tyl,
                                         const BwdSrcPair& s, BwdAcc& A) {
    const f2x dx = f2add(f2sub(tx, s.x), f2sub(txl, s.xl));
    const f2x dy = f2add(f2sub(ty, s.y), f2sub(tyl, s.yl));
    const f2x r2 = f2fma(dx, dx, f2fma(dy, dy, f2pk(1e-37f, 1e-37f)));
    float r0, r1;
    f2upk(r2, r0, r1);
    const f2x inv = f2pk(rcp_approx(r0), rcp_approx(r1));
    const f2x a = f2mul(dx, inv), b = f2mul(dy, inv);  // u = 1/d = a - i b
    const f2x ur = f2fma(a, a, f2mul(f2mul(b, b), f2pk(-1.f, -1.f)));  // u^2 = ur - i w
    const f2x b2 = f2add(b, b);
    const f2x w = f2mul(a, b2);                      // w = 2ab
    A.pr = f2fma(s.cr, a, f2fma(s.ci, b, A.pr));     // Re(c u)     = cr a + ci b
    A.pi = f2fma(s.ci, a, f2fma(s.ncr, b, A.pi));    // Im(c u)     = ci a - cr b
    A.qr = f2fma(s.ncr, ur, f2fma(s.nci, w, A.qr));  // Re(-c u^2)  = -cr ur - ci w
    A.qi = f2fma(s.nci, ur, f2fma(s.cr, w, A.qi));   // Im(-c u^2)  = -ci ur + cr w
    A.fr = f2fma(s.ngr, ur, f2fma(s.ngi, w, A.fr));  // Re(-g u^2)
    A.fi = f2fma(s.ngi, ur, f2fma(s.gr, w, A.fi));   // Im(-g u^2)
}

// One warp per P2P work item (the forward's items); lane (tg, ss) owns targets
// tg, tg + LT, ... (TPL of them) and slot-pair slice ss of S = 32/LT.  With
// LT = 4 a range (one strong entry) is one step of 2S = 16 slots; the other
// layouts take ceil(count/2S) steps per range.
constexpr int kBPWarps = 4;

template <int TPL, int LT>
__global__ void __launch_bounds__(kBPWarps * 32, 4)
    k_p2p_bwd_pairs(const int4* __restrict__ items, const unsigned long long* __restrict__ nitems,
                    const int32_t* __restrict__ bstart, const int32_t* __restrict__ bcount,
                    const int32_t* __restrict__ pslot, const int32_t* __restrict__ soff,
                    const int2* __restrict__ srng, const ulonglong2* __restrict__ posq,
                    const ulonglong2* __restrict__ gamq, const ulonglong2* __restrict__ cstq,
                    float2* __restrict__ nearv, float2* __restrict__ part, int n, long long part_stride, int TS,
                    const int32_t* __restrict__ rows, const unsigned long long* __restrict__ nheavy, long long cap) {
    constexpr int S = 32 / LT;
    constexpr bool LONG = LT > 4;
    const int lane = threadIdx.x & 31;
    const int tg = lane % LT, ss = lane / LT;
    const int nit = (int)*nitems;
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (row >= nit) return;  // warp-uniform
    const int it = p2p_row_item(row, rows, *nheavy, cap);  // the forward's row order: long items first
    const int4 item = items[it];
    const int b = item.x;
    const int ts = bstart[b], tn = bcount[b], tb = pslot[b];
    const int2* rl = srng + soff[b];
    for (int t0 = 0; t0 < tn; t0 += TPL * LT) {
        f2x tx[TPL], ty[TPL], txl[TPL], tyl[TPL];
        BwdAcc A[TPL];
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
            A[u] = BwdAcc{0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
        }
        if constexpr (!LONG) {
            // one step per range; the next range's sources are loaded while this one is computed
            int k = item.y;
            int q = ((k < item.z ? rl[k].x : 0) >> 1) + ss;
            ulonglong2 pa = posq[2 * q], pb = posq[2 * q + 1], ga = gamq[q], ca = cstq[q];
            for (; k < item.z; ++k) {
                const BwdSrcPair sp = bwd_src_pair(pa, pb, ga, ca);
                if (k + 1 < item.z) {
                    q = (rl[k + 1].x >> 1) + ss;
                    pa = posq[2 * q];
                    pb = posq[2 * q + 1];
                    ga = gamq[q];
                    ca = cstq[q];
                }
#pragma unroll
                for (int u = 0; u < TPL; ++u) bwd_pair(tx[u], ty[u], txl[u], tyl[u], sp, A[u]);
            }
        } else {
            for (int k = item.y; k < item.z; ++k) {
                const int2 r = rl[k];
                const int o = (r.x >> 1) + ss;  // slot-pair index of this slice
                const int steps = (r.y + 2 * S - 1) / (2 * S);
                for (int e = 0; e < steps; ++e) {
                    const int q = o + e * S;
                    const BwdSrcPair sp = bwd_src_pair(posq[2 * q], posq[2 * q + 1], gamq[q], cstq[q]);
#pragma unroll
                    for (int u = 0; u < TPL; ++u) bwd_pair(tx[u], ty[u], txl[u], tyl[u], sp, A[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < TPL; ++u) {
            float v[6];
            const f2x acc[6] = {A[u].pr, A[u].pi, A[u].qr, A[u].qi, A[u].fr, A[u].fi};
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                float lo, hi;
                f2upk(acc[c], lo, hi);
                v[c] = lo + hi;
#pragma unroll
                for (int off = LT; off < 32; off <<= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
            }
            const int idx = t0 + tg + u * LT;
            if (ss == 0 && idx < tn) {
                if (item.w < 0) {
                    nearv[ts + idx] = make_float2(v[0], v[1]);
                    nearv[(size_t)n + ts + idx] = make_float2(v[2], v[3]);
                    nearv[2 * (size_t)n + ts + idx] = make_float2(v[4], v[5]);
                } else {
                    const size_t qq = (size_t)it * TS + idx;
                    part[qq] = make_float2(v[0], v[1]);
                    part[part_stride + qq] = make_float2(v[2], v[3]);
                    part[2 * part_stride + qq] = make_float2(v[4], v[5]);
                }
            }
        }
    }
}

// ----------------------------------------------------------- near field

__device__ __forceinline__ void bwd_interact32(const float4 t, const float4 s, const float2 g, const float2 c,
                                               float2& psi, float2& dpsi, float2& dphi) {
    const float dx = (t.x - s.x) + (t.z - s.z);
    const float dy = (t.y - s.y) + (t.w - s.w);
    const float inv = fminf(rcp_approx(fmaf(dx, dx, dy * dy)), 3.0e38f);
    const float2 u = make_float2(dx * inv, -dy * inv);  // 1/(z_t - z_s); 0 for a coincident pair
    const float2 u2 = make_float2(fmaf(u.x, u.x, -u.y * u.y), 2.0f * u.x * u.y);
    psi = cfma(c, u, psi);
    dpsi = cfma(make_float2(-c.x, -c.y), u2, dpsi);
    dphi = cfma(make_float2(-g.x, -g.y), u2, dphi);
}

__device__ __forceinline__ void bwd_interact64(const double2 t, const double2 s, const double2 g, const double2 c,
                                               double2& psi, double2& dpsi, double2& dphi) {
    const double dx = t.x - s.x, dy = t.y - s.y;
    const double r2 = fma(dx, dx, dy * dy);
    const double inv = rcp_nr64(r2);  // 0 for a coincident pair
    const double2 u = make_double2(dx * inv, -dy * inv);
    const double2 u2 = make_double2(fma(u.x, u.x, -u.y * u.y), 2.0 * u.x * u.y);
    psi = cfma(c, u, psi);
    dpsi = cfma(make_double2(-c.x, -c.y), u2, dpsi);
    dphi = cfma(make_double2(-g.x, -g.y), u2, dphi);
}

// Same work decomposition as the forward P2P (one warp per item, lanes as
// target groups x source slices); three outputs per target.
template <typename V, typename C, int TPL, int CH>
__global__ void __launch_bounds__(kBWarps * 32) k_p2p_bwd(const int4* __restrict__ items,
                                                          const unsigned long long* __restrict__ nitems,
                                                          const int32_t* __restrict__ bstart,
                                                          const int32_t* __restrict__ bcount,
                                                          const int32_t* __restrict__ soff,
                                                          const int32_t* __restrict__ sidx, const V* __restrict__ pos,
                                                          const C* __restrict__ gam, const C* __restrict__ cst,
                                                          C* __restrict__ nearv, C* __restrict__ part, int n,
                                                          long long part_stride, int TS) {
    __shared__ V sp[kBWarps][CH];
    __shared__ C sg[kBWarps][CH];
    __shared__ C sc[kBWarps][CH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nit = (int)*nitems;
    for (int it = blockIdx.x * kBWarps + warp; it < nit; it += gridDim.x * kBWarps) {
        const int4 item = items[it];
        const int b = item.x;
        const int ts = bstart[b], tn = bcount[b];
        const int32_t* sl = sidx + soff[b];
        for (int t0 = 0; t0 < tn; t0 += 32 * TPL) {
            const int nt = min(tn - t0, 32 * TPL);
            const int LT = (nt + TPL - 1) / TPL;
            const int S = 32 / LT;
            const int tg = lane % LT, ss = lane / LT;
            const bool active = ss < S;
            V xt[TPL];
            C a0[TPL], a1[TPL], a2[TPL];
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
                const int idx = t0 + tg + u * LT;
                xt[u] = (idx < tn) ? pos[ts + idx] : V{};
                a0[u] = C{};
                a1[u] = C{};
                a2[u] = C{};
            }
            int j = item.y, off = 0;
            while (j < item.z) {
                __syncwarp();
                int cnt = 0;
                while (j < item.z && cnt < CH) {
                    const int h = sl[j];
                    const int hs = bstart[h], hn = bcount[h];
                    const int take = min(hn - off, CH - cnt);
                    for (int e = lane; e < take; e += 32) {
                        sp[warp][cnt + e] = pos[hs + off + e];
                        sg[warp][cnt + e] = gam[hs + off + e];
                        sc[warp][cnt + e] = cst[hs + off + e];
                    }
                    cnt += take;
                    off += take;
                    if (off == hn) {
                        ++j;
                        off = 0;
                    }
                }
                __syncwarp();
                if (active) {
                    for (int e = ss; e < cnt; e += S) {
                        const V s = sp[warp][e];
                        const C g = sg[warp][e], c = sc[warp][e];
#pragma unroll
                        for (int u = 0; u < TPL; ++u) {
                            if constexpr (sizeof(V) == 16 && sizeof(C) == 8)
                                bwd_interact32(xt[u], s, g, c, a0[u], a1[u], a2[u]);
                            else
                                bwd_interact64(xt[u], s, g, c, a0[u], a1[u], a2[u]);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
                C t0v = a0[u], t1v = a1[u], t2v = a2[u];
                for (int s2 = 1; s2 < S; ++s2) {
                    const int src = (tg + s2 * LT) & 31;
                    t0v.x += __shfl_sync(0xffffffffu, a0[u].x, src);
                    t0v.y += __shfl_sync(0xffffffffu, a0[u].y, src);
                    t1v.x += __shfl_sync(0xffffffffu, a1[u].x, src);
                    t1v.y += __shfl_sync(0xffffffffu, a1[u].y, src);
                    t2v.x += __shfl_sync(0xffffffffu, a2[u].x, src);
                    t2v.y += __shfl_sync(0xffffffffu, a2[u].y, src);
                }
                const int idx = t0 + tg + u * LT;
                if (ss == 0 && idx < tn) {
                    if (item.w < 0) {
                        nearv[ts + idx] = t0v;
                        nearv[(size_t)n + ts + idx] = t1v;
                        nearv[2 * (size_t)n + ts + idx] = t2v;
                    } else {
                        const size_t q = (size_t)it * TS + idx;
                        part[q] = t0v;
                        part[part_stride + q] = t1v;
                        part[2 * part_stride + q] = t2v;
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------- L2P + assembly

template <typename C>
__device__ __forceinline__ C near_sum(int i, int r, int ls, int2 li, const C* __restrict__ nearv,
                                      const C* __restrict__ part, int n, long long stride, int TS) {
    if (li.y == 1) return nearv[(size_t)r * n + i];
    C s{};
    for (int q = 0; q < li.y; ++q) {
        const C v = part[r * stride + (size_t)(li.x + q) * TS + (i - ls)];
        s.x += v.x;
        s.y += v.y;
    }
    return s;
}

// value and z-derivative of sum_l b_l w^l, w = (z-c)/rho: dL/dz = (dL/dw)/rho
template <int P, typename C, typename R>
__device__ __forceinline__ void horner2(const C* __restrict__ b, C w, R inv, C& v, C& dv) {
    v = b[P - 1];
    dv = C{};
#pragma unroll
    for (int l = P - 2; l >= 0; --l) {
        dv = cfma(dv, w, v);
        v = cfma(v, w, b[l]);
    }
    dv.x *= inv;
    dv.y *= inv;
}

// horner2 over the terms l < p only (a box's own M2L sum holds P terms).
template <int P>
__device__ __forceinline__ void horner2_p(const float2* __restrict__ b, float2 w, float inv, int p, float2& v,
                                          float2& dv) {
    v = P - 1 < p ? b[P - 1] : make_float2(0.f, 0.f);
    dv = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = P - 2; l >= 0; --l) {
        dv = cfma(dv, w, v);
        v = cfma(v, w, l < p ? b[l] : make_float2(0.f, 0.f));
    }
    dv.x *= inv;
    dv.y *= inv;
}

// Far field (value and z-derivative) of a leaf of the deepest level on the
// FP32 path, which has no shifted local: the parent's local and the leaf's own
// M2L sum, each at the point.
template <int P>
__device__ __forceinline__ void far_folded(const float4 pt, int par, int lf, const float4* __restrict__ chl,
                                           const float* __restrict__ rho32, const float2* __restrict__ L,
                                           const float2* __restrict__ M, bool own, int p, int PS, float2& v,
                                           float2& dv) {
    const float4 c = chl[par];
    const float r = rho32[par];
    const float inv = r > 0.f ? 1.0f / r : 0.f;
    const float2 w = make_float2(((pt.x - c.x) + (pt.z - c.z)) * inv, ((pt.y - c.y) + (pt.w - c.w)) * inv);
    horner2<P>(L + (size_t)par * PS, w, inv, v, dv);
    if (own) {
        const float4 cl = chl[lf];
        const float rl = rho32[lf];
        const float il = rl > 0.f ? 1.0f / rl : 0.f;
        const float2 wl = make_float2(((pt.x - cl.x) + (pt.z - cl.z)) * il, ((pt.y - cl.y) + (pt.w - cl.w)) * il);
        float2 ov, odv;
        horner2_p<P>(M + (size_t)lf * PS, wl, il, p, ov, odv);
        v.x += ov.x;
        v.y += ov.y;
        dv.x += odv.x;
        dv.y += odv.y;
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_l2p_bwd32(int n, const int32_t* __restrict__ leaf_of,
                                                   const int32_t* __restrict__ fold_par,
                                                   const int2* __restrict__ box_m2l,
                                                   const int32_t* __restrict__ bstart, const float4* __restrict__ chl,
                                                   const float* __restrict__ rho32, const float4* __restrict__ pos4,
                                                   const float2* __restrict__ Lg, const float2* __restrict__ Lc,
                                                   const float2* __restrict__ Mg, const float2* __restrict__ Mc,
                                                   const int2* __restrict__ leaf_items,
                                                   const float2* __restrict__ nearv, const float2* __restrict__ part,
                                                   long long stride, int TS, const int32_t* __restrict__ perm,
                                                   const double2* __restrict__ gam, const double2* __restrict__ gphi,
                                                   double2* __restrict__ ggam, double2* __restrict__ gxy, int p,
                                                   int PS) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf_of[i];
    const float4 pt = pos4[i];
    const int par = fold_par[lf];
    float2 vg, dphi, psi, dpsi;
    if (par >= 0) {
        const bool own = box_m2l[lf].y > 0;
        far_folded<P>(pt, par, lf, chl, rho32, Lg, Mg, own, p, PS, vg, dphi);
        far_folded<P>(pt, par, lf, chl, rho32, Lc, Mc, own, p, PS, psi, dpsi);
    } else {
        const float4 c = chl[lf];
        const float r = rho32[lf];
        const float inv = r > 0.f ? 1.0f / r : 0.f;
        const float2 w = make_float2(((pt.x - c.x) + (pt.z - c.z)) * inv, ((pt.y - c.y) + (pt.w - c.w)) * inv);
        horner2<P>(Lg + (size_t)lf * PS, w, inv, vg, dphi);
        horner2<P>(Lc + (size_t)lf * PS, w, inv, psi, dpsi);
    }
    const int ls = bstart[lf];
    const int2 li = leaf_items[lf];
    const float2 n0 = near_sum(i, 0, ls, li, nearv, part, n, stride, TS);
    const float2 n1 = near_sum(i, 1, ls, li, nearv, part, n, stride, TS);
    const float2 n2 = near_sum(i, 2, ls, li, nearv, part, n, stride, TS);
    const double2 Psi = make_double2((double)psi.x + n0.x, (double)psi.y + n0.y);
    const double2 dPsi = make_double2((double)dpsi.x + n1.x, (double)dpsi.y + n1.y);
    const double2 dPhi = make_double2((double)dphi.x + n2.x, (double)dphi.y + n2.y);
    const int o = perm[i];
    const double2 g = gam[o], u = gphi[o];
    const double2 ck = make_double2(u.x, -u.y);
    const double2 D = cfma(ck, dPhi, cmul(make_double2(-g.x, -g.y), dPsi));
    if (ggam) ggam[o] = make_double2(-Psi.x, Psi.y);
    if (gxy) gxy[o] = make_double2(D.x, -D.y);
}

template <int P>
__global__ void __launch_bounds__(256) k_l2p_bwd64(int n, const int32_t* __restrict__ leaf_of,
                                                   const int32_t* __restrict__ bstart,
                                                   const double2* __restrict__ center, const double* __restrict__ rho,
                                                   const double2* __restrict__ pts, const double2* __restrict__ Lg,
                                                   const double2* __restrict__ Lc,
                                                   const int2* __restrict__ leaf_items,
                                                   const double2* __restrict__ nearv,
                                                   const double2* __restrict__ part, long long stride, int TS,
                                                   const int32_t* __restrict__ perm, const double2* __restrict__ gam,
                                                   const double2* __restrict__ gphi, double2* __restrict__ ggam,
                                                   double2* __restrict__ gxy, int PS) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lf = leaf_of[i];
    const double2 c = center[lf];
    const double r = rho[lf];
    const double inv = r > 0.0 ? 1.0 / r : 0.0;
    const double2 pt = pts[i];
    const double2 w = make_double2((pt.x - c.x) * inv, (pt.y - c.y) * inv);
    double2 vg, dphi, psi, dpsi;
    horner2<P>(Lg + (size_t)lf * PS, w, inv, vg, dphi);
    horner2<P>(Lc + (size_t)lf * PS, w, inv, psi, dpsi);
    const int ls = bstart[lf];
    const int2 li = leaf_items[lf];
    const double2 n0 = near_sum(i, 0, ls, li, nearv, part, n, stride, TS);
    const double2 n1 = near_sum(i, 1, ls, li, nearv, part, n, stride, TS);
    const double2 n2 = near_sum(i, 2, ls, li, nearv, part, n, stride, TS);
    const double2 Psi = make_double2(psi.x + n0.x, psi.y + n0.y);
    const double2 dPsi = make_double2(dpsi.x + n1.x, dpsi.y + n1.y);
    const double2 dPhi = make_double2(dphi.x + n2.x, dphi.y + n2.y);
    const int o = perm[i];
    const double2 g = gam[o], u = gphi[o];
    const double2 ck = make_double2(u.x, -u.y);
    const double2 D = cfma(ck, dPhi, cmul(make_double2(-g.x, -g.y), dPsi));
    if (ggam) ggam[o] = make_double2(-Psi.x, Psi.y);
    if (gxy) gxy[o] = make_double2(D.x, -D.y);
}

#define FMM_BWD_ORDERS(X) X(4) X(8) X(12) X(16) X(17) X(20) X(24) X(28) X(32)

template <int P>
static void launch_l2p_bwd(Tree& t, const Bufs& B0, const Bufs& B1, const double* d_gamma, const double* d_gphi,
                           double* d_ggamma, double* d_gxy, cudaStream_t s) {
    const int n = (int)t.n;
    const long long stride = (long long)t.part_p2p_cap * t.max_leaf;
    const double2* gam = reinterpret_cast<const double2*>(d_gamma);
    const double2* gph = reinterpret_cast<const double2*>(d_gphi);
    double2* gg = reinterpret_cast<double2*>(d_ggamma);
    double2* gx = reinterpret_cast<double2*>(d_gxy);
    if (t.path == FMM_PATH_FP32)
        k_l2p_bwd32<P><<<nblk(n, 256), 256, 0, s>>>(
            n, t.d_leaf_of, t.d_fold_par, t.d_box_m2l, t.d_bstart, t.d_chl, t.d_rho32, t.d_pos4, B0.L32, B1.L32,
            static_cast<const float2*>(B0.Lm2l), static_cast<const float2*>(B1.Lm2l), t.d_leaf_items,
            static_cast<const float2*>(t.d_near), static_cast<const float2*>(t.d_p2p_part), stride, t.max_leaf,
            t.d_perm, gam, gph, gg, gx, t.p, t.PS);
    else
        k_l2p_bwd64<P><<<nblk(n, 256), 256, 0, s>>>(n, t.d_leaf_of, t.d_bstart, t.d_center, t.d_rho, t.d_pts,
                                                    B0.L64, B1.L64, t.d_leaf_items,
                                                    static_cast<const double2*>(t.d_near),
                                                    static_cast<const double2*>(t.d_p2p_part), stride, t.max_leaf,
                                                    t.d_perm, gam, gph, gg, gx, t.PS);
}

fmm_status run_backward(Tree& t, const double* d_gamma, const double* d_gphi, double* d_ggamma, double* d_gxy,
                        cudaStream_t s) {
    const int n = (int)t.n;
    const Bufs B0 = bufs(t, 0), B1 = bufs(t, 1);
    const double2* gin = reinterpret_cast<const double2*>(d_gamma);
    const double2* pin = reinterpret_cast<const double2*>(d_gphi);
    const bool f32 = t.path == FMM_PATH_FP32;
    if (f32) {
        // the second strength set in the slot layout (padding slots stay zero)
        if (t.gamp2_slots != t.slot_alloc) {
            if (t.d_gamp2) cudaFree(t.d_gamp2);
            t.d_gamp2 = nullptr;
            t.gamp2_slots = 0;
            FMM_CUDA(cudaMalloc(&t.d_gamp2, (size_t)std::max<int64_t>(t.slot_alloc, 1) * sizeof(float2)));
            FMM_CUDA(cudaMemsetAsync(t.d_gamp2, 0, (size_t)std::max<int64_t>(t.slot_alloc, 1) * sizeof(float2), s));
            t.gamp2_slots = t.slot_alloc;
        }
        k_gather_bwd<float2><<<nblk(n, 256), 256, 0, s>>>(gin, pin, t.d_perm, t.d_slot_of, n,
                                                          static_cast<float2*>(B0.gam), static_cast<float2*>(B1.gam),
                                                          static_cast<float*>(t.d_gamp),
                                                          static_cast<float*>(t.d_gamp2));
    } else {
        k_gather_bwd<double2><<<nblk(n, 256), 256, 0, s>>>(gin, pin, t.d_perm, t.d_slot_of, n,
                                                           static_cast<double2*>(B0.gam),
                                                           static_cast<double2*>(B1.gam), nullptr, nullptr);
    }
    FMM_CUDA(cudaEventRecord(t.ev_fork, s));
    FMM_CUDA(cudaStreamWaitEvent(t.s_aux, t.ev_fork, 0));
    FMM_CUDA(cudaStreamWaitEvent(t.s_far2, t.ev_fork, 0));
    const int grid = nblk(p2p_grid_items(t), kBWarps);
    const long long stride = (long long)t.part_p2p_cap * t.max_leaf;
    const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(t.d_status) + 3;
    const bool wide = (double)t.n / std::max<int64_t>(t.nleaf, 1) >= 8.0;
    if (f32) {
        // packed f32x2 over the forward's slot layout, half the forward's targets per lane (three sums each)
        auto* nv = static_cast<float2*>(t.d_near);
        auto* pt = static_cast<float2*>(t.d_p2p_part);
        const int pgrid = nblk(p2p_grid_items(t), kBPWarps);
        const P2PLayout pl = p2p_pair_layout(t.max_leaf);
        const auto* pq = static_cast<const ulonglong2*>(t.d_posp);
        const auto* gq = static_cast<const ulonglong2*>(t.d_gamp);
        const auto* cq = static_cast<const ulonglong2*>(t.d_gamp2);
#define FMM_BWD_PAIRS(TPL, LT)                                                                                   \
    k_p2p_bwd_pairs<TPL, LT><<<pgrid, kBPWarps * 32, 0, t.s_aux>>>(t.d_p2p_items, cnt, t.d_bstart, t.d_bcount,  \
                                                                    t.d_pslot, t.d_soff, t.d_srng, pq, gq, cq, nv, \
                                                                    pt, n, stride, t.max_leaf, t.d_p2p_rows,       \
                                                                    t.d_m2l_rowctr + kM2LItemPairsMax + 1, t.p2p_cap);
        switch (pl.tpl * 100 + pl.lt) {
            case 204: FMM_BWD_PAIRS(1, 4) break;
            case 404: FMM_BWD_PAIRS(2, 4) break;
            case 408: FMM_BWD_PAIRS(2, 8) break;
            case 416: FMM_BWD_PAIRS(2, 16) break;
            default: FMM_BWD_PAIRS(4, 16) break;
        }
#undef FMM_BWD_PAIRS
        (void)wide;
    } else {
        auto* g = static_cast<const double2*>(B0.gam);
        auto* c = static_cast<const double2*>(B1.gam);
        auto* nv = static_cast<double2*>(t.d_near);
        auto* pt = static_cast<double2*>(t.d_p2p_part);
        if (wide)
            k_p2p_bwd<double2, double2, 4, kBChunk64><<<grid, kBWarps * 32, 0, t.s_aux>>>(
                t.d_p2p_items, cnt, t.d_bstart, t.d_bcount, t.d_soff, t.d_sidx, t.d_pts, g, c, nv, pt, n, stride,
                t.max_leaf);
        else
            k_p2p_bwd<double2, double2, 1, kBChunk64><<<grid, kBWarps * 32, 0, t.s_aux>>>(
                t.d_p2p_items, cnt, t.d_bstart, t.d_bcount, t.d_soff, t.d_sidx, t.d_pts, g, c, nv, pt, n, stride,
                t.max_leaf);
    }
    FMM_CUDA(cudaEventRecord(t.ev_join, t.s_aux));
    const int flags = t.flags;
    t.flags &= ~FMM_FLAG_TIMING;
    // the two strength sets' far fields side by side (latency-bound kernels overlap)
    dispatch_far(t, B0, s);
    dispatch_far(t, B1, t.s_far2);
    t.flags = flags;
    FMM_CUDA(cudaEventRecord(t.ev_join_far2, t.s_far2));
    FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join_far2, 0));
    FMM_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
    switch (t.P) {
#define FMM_CASE(Q) \
    case Q: launch_l2p_bwd<Q>(t, B0, B1, d_gamma, d_gphi, d_ggamma, d_gxy, s); break;
        FMM_BWD_ORDERS(FMM_CASE)
#undef FMM_CASE
    }
    FMM_CUDA(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmm
