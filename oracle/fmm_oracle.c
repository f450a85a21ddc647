/*
 * fmm_oracle.c -- the ORACLE for the balanced adaptive 2D FMM (harmonic kernel).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct CPU
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the library's
 * product path never calls it, and it shares no code, header, table or helper
 * with the CUDA sources.
 *
 * Method: Holm, Engblom, Goude, Holmgren, "Dynamic autotuning of adaptive fast
 * multipole methods on hybrid multicore CPU & GPU systems" (arXiv:1311.1006).
 *
 *   Problem (Sec. 2, eq 2.1 / 2.2, harmonic kernel of Sec. 3.3, sign +):
 *       Phi(z_i) = sum_{j : z_j != z_i} Gamma_j / (z_i - z_j),  z = x + i y complex.
 *   Tree (Sec. 2.2-2.3): pyramid of N_levels full levels, N_f = 4^(N_levels-1)
 *       leaves; every box is split into 4 children at medians (x first, then y
 *       in each half), so every leaf holds ~N/N_f points.
 *   Coupling (Sec. 2.1, eq 2.3): theta-criterion  R + theta*r <= theta*d;
 *       strong / weak / decoupled pairs per level.
 *   Passes (Sec. 2.1, Fig 2.2): P2M, M2M (upward), M2L + L2L (downward),
 *       L2P and P2P at the finest level.
 *
 * The paper prints no expansion formulas for the harmonic kernel, so this
 * oracle uses the textbook Cauchy-kernel series written out from their
 * definitions, with UNSCALED coefficients (the GPU uses radius-scaled ones; the
 * two formulations are independent):
 *   multipole about c:  M(z) = sum_{k<p} a_k / (z-c)^(k+1),   a_k = sum_j Gamma_j (z_j-c)^k
 *   local about c:      L(z) = sum_{l<p} b_l (z-c)^l
 *   M2M  a'_n = sum_{k<=n} C(n,k) a_k s^(n-k),            s = c_child - c_parent
 *   M2L  b_l += (-1)^l sum_k C(k+l,l) a_k / d^(k+l+1),    d = c_target - c_source
 *   L2L  b'_m = sum_{l>=m} C(l,m) b_l s^(l-m),            s = c_child - c_parent
 *   L2P  Phi_far(z) = sum_l b_l (z-c)^l,  Phi_far'(z) = sum_l l b_l (z-c)^(l-1)
 *   P2P  Phi_near(z_i) = sum over points j of the strongly coupled leaves,
 *        z_j != z_i, of Gamma_j/(z_i-z_j);  derivative -Gamma_j/(z_i-z_j)^2.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *   R1  kernel sign +Gamma_j/(z_i-z_j) (the paper's harmonic kernel has a minus;
 *       a global factor).
 *   R2  "p terms" = coefficients k = 0..p-1 in both expansions.
 *   R3  split = exact ranks: sort a box by (x, original index), lower floor(n/2)
 *       points go left; sort each half by (y, original index), lower floor(m/2)
 *       go to the bottom.  Children 0..3 = (left,bottom),(left,top),
 *       (right,bottom),(right,top).  Points inside a leaf are ordered by
 *       (y, original index).
 *   R4  box geometry = tight bounding box of its points: centre = midpoint,
 *       radius = half the diagonal.
 *   R5  theta-test: d = |c_1 - c_2|, equality counts as well separated, and a
 *       pair with d == 0 is never well separated (the M2L series is singular).
 *   R6  level 0 is the root, strongly coupled with itself only.
 *   R7  pairs with z_j == z_i contribute nothing (eq 2.2's exclusion).
 *
 * Box numbering: level l holds 4^l boxes; box b of level l has the global id
 * (4^l - 1)/3 + b and children 4b..4b+3 on level l+1.
 * Complex arrays are interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ utils */

static int g_threads = 0; /* 0 = library default */

void fo_set_threads(int t) {
    g_threads = t;
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#endif
}

int fo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int64_t fo_num_boxes(int nlevels) {
    int64_t s = 0, w = 1;
    for (int l = 0; l < nlevels; ++l) { s += w; w *= 4; }
    return s;
}

static int64_t level_offset(int l) { return fo_num_boxes(l); }

static cplx load_c(const double* a, int64_t i) { return a[2 * i] + I * a[2 * i + 1]; }
static void store_c(double* a, int64_t i, cplx v) { a[2 * i] = creal(v); a[2 * i + 1] = cimag(v); }

/* Binomial coefficient C(n,k) from Pascal's rule, exact in FP64 for n <= 56. */
static double binom(int n, int k) {
    static double tab[80][80];
    static int ready = 0;
    if (!ready) {
        for (int a = 0; a < 80; ++a) {
            tab[a][0] = 1.0;
            for (int b = 1; b <= a; ++b) tab[a][b] = tab[a - 1][b - 1] + (b <= a - 1 ? tab[a - 1][b] : 0.0);
            for (int b = a + 1; b < 80; ++b) tab[a][b] = 0.0;
        }
        ready = 1;
    }
    if (k < 0 || k > n) return 0.0;
    return tab[n][k];
}


/* z^e for e >= 0 by repeated multiplication (0^0 = 1). */
static cplx cpow_int(cplx z, int e) {
    cplx r = 1;
    for (int i = 0; i < e; ++i) r *= z;
    return r;
}

/* ------------------------------------------------------------ direct sums */

/* Exact sum of eq (2.2) at the targets tgt[0..m) (all n points when tgt == NULL):
 *   phi[t]  = sum_{z_j != z_t} Gamma_j / (z_t - z_j)
 *   dphi[t] = d/dz of the same = - sum Gamma_j / (z_t - z_j)^2     (optional)  */
void fo_direct(int64_t n, const double* xy, const double* gam, int64_t m, const int64_t* tgt,
               double* phi, double* dphi) {
    if (tgt == NULL) m = n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        int64_t t = tgt ? tgt[q] : q;
        cplx zt = xy[2 * t] + I * xy[2 * t + 1];
        cplx s = 0, ds = 0;
        for (int64_t j = 0; j < n; ++j) {
            cplx zj = xy[2 * j] + I * xy[2 * j + 1];
            if (zj == zt) continue; /* R7 */
            cplx r = 1.0 / (zt - zj);
            s += load_c(gam, j) * r;
            ds -= load_c(gam, j) * r * r;
        }
        store_c(phi, q, s);
        if (dphi) store_c(dphi, q, ds);
    }
}

/* Exact sum of eq (2.2) with separate evaluation points: for each of the m
 * points y_t (txy, interleaved x, y), phi[t] = sum_{j: x_j != y_t} Gamma_j / (y_t - x_j)
 * over the n sources x_j (sxy).                                                      */
void fo_direct_points(int64_t n, const double* sxy, const double* gam, int64_t m, const double* txy, double* phi) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < m; ++t) {
        cplx yt = txy[2 * t] + I * txy[2 * t + 1];
        cplx s = 0;
        for (int64_t j = 0; j < n; ++j) {
            cplx xj = sxy[2 * j] + I * sxy[2 * j + 1];
            if (xj == yt) continue; /* eq (2.2): x_j != y_t */
            s += load_c(gam, j) / (yt - xj);
        }
        store_c(phi, t, s);
    }
}

/* Exact gradient of the loss  L = sum_i w_i Re Phi_i + v_i Im Phi_i  with
 * upstream gphi_i = w_i + i v_i, at the points tgt[0..m) (all when NULL).
 * Derivation (chain rule on the holomorphic kernel), with c_i = conj(gphi_i):
 *   L = Re sum_i c_i Phi_i
 *   dL/dRe Gamma_k + i dL/dIm Gamma_k = -conj(Psi_k),  Psi_k = sum_{i: z_i!=z_k} c_i/(z_k - z_i)
 *   D_k = c_k Phi'_k - Gamma_k Psi'_k,  Phi'_k = -sum Gamma_j/(z_k-z_j)^2,  Psi'_k = -sum c_i/(z_k-z_i)^2
 *   dL/dx_k = Re D_k,   dL/dy_k = -Im D_k.                                      */
void fo_direct_grad(int64_t n, const double* xy, const double* gam, const double* gphi, int64_t m,
                    const int64_t* tgt, double* ggam, double* gxy) {
    if (tgt == NULL) m = n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        int64_t k = tgt ? tgt[q] : q;
        cplx zk = xy[2 * k] + I * xy[2 * k + 1];
        cplx psi = 0, dpsi = 0, dphi = 0;
        for (int64_t j = 0; j < n; ++j) {
            cplx zj = xy[2 * j] + I * xy[2 * j + 1];
            if (zj == zk) continue;
            cplx r = 1.0 / (zk - zj);
            cplx cj = conj(load_c(gphi, j));
            psi += cj * r;
            dpsi -= cj * r * r;
            dphi -= load_c(gam, j) * r * r;
        }
        cplx ck = conj(load_c(gphi, k));
        cplx D = ck * dphi - load_c(gam, k) * dpsi;
        store_c(ggam, q, -conj(psi));
        gxy[2 * q] = creal(D);
        gxy[2 * q + 1] = -cimag(D);
    }
}

/* ------------------------------------------------------------------- tree */

typedef struct { double key; int64_t idx; } keyed;

static int cmp_keyed(const void* a, const void* b) {
    const keyed* u = (const keyed*)a;
    const keyed* v = (const keyed*)b;
    if (u->key < v->key) return -1;
    if (u->key > v->key) return 1;
    return (u->idx > v->idx) - (u->idx < v->idx);
}

/* Sort ids[0..n) by (coordinate dim, original index). */
static void sort_by(int64_t* ids, int64_t n, const double* xy, int dim, keyed* tmp) {
    for (int64_t i = 0; i < n; ++i) { tmp[i].key = xy[2 * ids[i] + dim]; tmp[i].idx = ids[i]; }
    qsort(tmp, (size_t)n, sizeof(keyed), cmp_keyed);
    for (int64_t i = 0; i < n; ++i) ids[i] = tmp[i].idx;
}

/* Build the pyramid tree (Sec. 2.2-2.3, readings R3/R4).
 *   perm[n]        : sorted position -> original point index
 *   bstart, bcount : per global box id, the range of its points in perm
 *   center[2*nb]   : box centre (x, y);  radius[nb] : half diagonal of the bbox
 * Returns 0, or -1 when nlevels < 1 or 4^(nlevels-1) > n (empty leaves).       */
int fo_build_tree(int64_t n, const double* xy, int nlevels, int64_t* perm, int64_t* bstart,
                  int64_t* bcount, double* center, double* radius) {
    if (nlevels < 1 || n < 1) return -1;
    if (fo_num_boxes(nlevels) - fo_num_boxes(nlevels - 1) > n) return -1;
    keyed* tmp = (keyed*)malloc(sizeof(keyed) * (size_t)n);
    if (!tmp) return -2;
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    bstart[0] = 0;
    bcount[0] = n;
    for (int l = 0; l + 1 < nlevels; ++l) {
        int64_t nb = fo_num_boxes(l + 1) - fo_num_boxes(l);
        for (int64_t b = 0; b < nb; ++b) {
            int64_t g = level_offset(l) + b;
            int64_t s = bstart[g], cnt = bcount[g];
            int64_t* ids = perm + s;
            int64_t nl = cnt / 2, nr = cnt - nl;
            sort_by(ids, cnt, xy, 0, tmp);      /* x-median split */
            sort_by(ids, nl, xy, 1, tmp);       /* left half by y */
            sort_by(ids + nl, nr, xy, 1, tmp);  /* right half by y */
            int64_t c0 = level_offset(l + 1) + 4 * b;
            bstart[c0 + 0] = s;            bcount[c0 + 0] = nl / 2;
            bstart[c0 + 1] = s + nl / 2;   bcount[c0 + 1] = nl - nl / 2;
            bstart[c0 + 2] = s + nl;       bcount[c0 + 2] = nr / 2;
            bstart[c0 + 3] = s + nl + nr / 2; bcount[c0 + 3] = nr - nr / 2;
        }
    }
    /* R3: inside each leaf the order is (y, index); a no-op unless nlevels == 1. */
    {
        int64_t l0 = level_offset(nlevels - 1), nb = fo_num_boxes(nlevels) - l0;
        for (int64_t b = 0; b < nb; ++b) sort_by(perm + bstart[l0 + b], bcount[l0 + b], xy, 1, tmp);
    }
    /* R4: tight bbox of every box. */
    int64_t nbox = fo_num_boxes(nlevels);
    for (int64_t g = 0; g < nbox; ++g) {
        double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
        for (int64_t i = bstart[g]; i < bstart[g] + bcount[g]; ++i) {
            double x = xy[2 * perm[i]], y = xy[2 * perm[i] + 1];
            if (x < x0) x0 = x;
            if (x > x1) x1 = x;
            if (y < y0) y0 = y;
            if (y > y1) y1 = y;
        }
        double dx = x1 - x0, dy = y1 - y0;
        center[2 * g] = 0.5 * (x0 + x1);
        center[2 * g + 1] = 0.5 * (y0 + y1);
        radius[g] = 0.5 * sqrt(dx * dx + dy * dy);
    }
    free(tmp);
    return 0;
}

/* --------------------------------------------------------------- coupling */

/* eq (2.3) with readings R5: R + theta*r <= theta*d and d > 0. */
static int well_separated(const double* center, const double* radius, int64_t a, int64_t b, double theta) {
    double dx = center[2 * a] - center[2 * b];
    double dy = center[2 * a + 1] - center[2 * b + 1];
    double d = sqrt(dx * dx + dy * dy);
    double R = radius[a] > radius[b] ? radius[a] : radius[b];
    double r = radius[a] > radius[b] ? radius[b] : radius[a];
    return d > 0.0 && R + theta * r <= theta * d;
}

static int cmp_i32(const void* a, const void* b) {
    int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
    return (u > v) - (u < v);
}

/* Strong / weak lists of every box (Sec. 2.1): a box is strong with itself;
 * children of strongly coupled boxes are strong unless they pass the
 * theta-test, in which case they are weak; children of weak pairs are
 * decoupled.  Lists hold global box ids, sorted ascending per box.
 * Two-call protocol: with s_idx == NULL only the CSR offsets s_off/w_off
 * (nbox+1 entries each) are written; the second call fills the lists.        */
int fo_build_lists(int nlevels, const double* center, const double* radius, double theta, int64_t* s_off,
                   int64_t* w_off, int32_t* s_idx, int32_t* w_idx) {
    int64_t nbox = fo_num_boxes(nlevels);
    /* working lists, one dynamic array per box */
    int32_t** S = (int32_t**)calloc((size_t)nbox, sizeof(int32_t*));
    int32_t** W = (int32_t**)calloc((size_t)nbox, sizeof(int32_t*));
    int64_t* ns = (int64_t*)calloc((size_t)nbox, sizeof(int64_t));
    int64_t* nw = (int64_t*)calloc((size_t)nbox, sizeof(int64_t));
    if (!S || !W || !ns || !nw) return -2;
    S[0] = (int32_t*)malloc(sizeof(int32_t));
    S[0][0] = 0;
    ns[0] = 1;
    for (int l = 1; l < nlevels; ++l) {
        int64_t off = level_offset(l), poff = level_offset(l - 1);
        int64_t nb = fo_num_boxes(l + 1) - off;
        for (int64_t b = 0; b < nb; ++b) {
            int64_t g = off + b;
            int64_t P = poff + b / 4;
            int64_t cap = 4 * ns[P];
            S[g] = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
            W[g] = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
            for (int64_t q = 0; q < ns[P]; ++q) {
                int64_t Q = S[P][q] - poff; /* index of the coupled parent within level l-1 */
                for (int c = 0; c < 4; ++c) {
                    int64_t h = off + 4 * Q + c;
                    if (h == g) S[g][ns[g]++] = (int32_t)h;
                    else if (well_separated(center, radius, g, h, theta)) W[g][nw[g]++] = (int32_t)h;
                    else S[g][ns[g]++] = (int32_t)h;
                }
            }
            qsort(S[g], (size_t)ns[g], sizeof(int32_t), cmp_i32);
            qsort(W[g], (size_t)nw[g], sizeof(int32_t), cmp_i32);
        }
    }
    s_off[0] = 0;
    w_off[0] = 0;
    for (int64_t g = 0; g < nbox; ++g) {
        s_off[g + 1] = s_off[g] + ns[g];
        w_off[g + 1] = w_off[g] + nw[g];
        if (s_idx) memcpy(s_idx + s_off[g], S[g], sizeof(int32_t) * (size_t)ns[g]);
        if (w_idx && nw[g]) memcpy(w_idx + w_off[g], W[g], sizeof(int32_t) * (size_t)nw[g]);
        free(S[g]);
        free(W[g]);
    }
    free(S); free(W); free(ns); free(nw);
    return 0;
}

/* ------------------------------------------------------------------ passes */

/* P2M on every leaf:  a_k = sum_{j in box} Gamma_j (z_j - c)^k. */
void fo_p2m(int nlevels, int p, const double* xy, const double* gam, const int64_t* perm, const int64_t* bstart,
            const int64_t* bcount, const double* center, double* mpole) {
    int64_t l0 = level_offset(nlevels - 1), nb = fo_num_boxes(nlevels) - l0;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t g = l0 + b;
        cplx c = center[2 * g] + I * center[2 * g + 1];
        for (int k = 0; k < p; ++k) store_c(mpole, g * p + k, 0);
        for (int64_t i = bstart[g]; i < bstart[g] + bcount[g]; ++i) {
            int64_t j = perm[i];
            cplx w = (xy[2 * j] + I * xy[2 * j + 1]) - c;
            cplx t = load_c(gam, j);
            for (int k = 0; k < p; ++k) {
                store_c(mpole, g * p + k, load_c(mpole, g * p + k) + t);
                t *= w;
            }
        }
    }
}

/* M2M, finest-but-one level up to the root:
 *   a'_n(parent) = sum_children sum_{k<=n} C(n,k) a_k(child) s^(n-k).        */
void fo_m2m(int nlevels, int p, const double* center, double* mpole) {
    for (int l = nlevels - 2; l >= 0; --l) {
        int64_t off = level_offset(l), nb = fo_num_boxes(l + 1) - off;
#pragma omp parallel for schedule(static)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t g = off + b;
            cplx cp = center[2 * g] + I * center[2 * g + 1];
            for (int n = 0; n < p; ++n) store_c(mpole, g * p + n, 0);
            for (int c = 0; c < 4; ++c) {
                int64_t h = level_offset(l + 1) + 4 * b + c;
                cplx s = (center[2 * h] + I * center[2 * h + 1]) - cp;
                for (int n = 0; n < p; ++n) {
                    cplx acc = 0;
                    for (int k = 0; k <= n; ++k) acc += binom(n, k) * load_c(mpole, h * p + k) * cpow_int(s, n - k);
                    store_c(mpole, g * p + n, load_c(mpole, g * p + n) + acc);
                }
            }
        }
    }
}

/* M2L into every box of levels 1..nlevels-1 from its weak list (eq 2.5 shift):
 *   b_l += (-1)^l sum_k C(k+l,l) a_k(src) / d^(k+l+1),  d = c_tgt - c_src.     */
void fo_m2l(int nlevels, int p, const double* center, const int64_t* w_off, const int32_t* w_idx,
            const double* mpole, double* local) {
    int64_t nbox = fo_num_boxes(nlevels);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < nbox; ++g) {
        cplx ct = center[2 * g] + I * center[2 * g + 1];
        for (int l = 0; l < p; ++l) store_c(local, g * p + l, 0);
        for (int64_t q = w_off[g]; q < w_off[g + 1]; ++q) {
            int64_t h = w_idx[q];
            cplx d = ct - (center[2 * h] + I * center[2 * h + 1]);
            cplx dinv[130]; /* dinv[m] = 1/d^m */
            dinv[0] = 1;
            for (int m = 1; m <= 2 * p; ++m) dinv[m] = dinv[m - 1] / d;
            for (int l = 0; l < p; ++l) {
                cplx acc = 0;
                for (int k = 0; k < p; ++k) acc += binom(k + l, l) * load_c(mpole, h * p + k) * dinv[k + l + 1];
                if (l & 1) acc = -acc;
                store_c(local, g * p + l, load_c(local, g * p + l) + acc);
            }
        }
    }
}

/* L2L, root down to the leaves:  b'_m(child) += sum_{l>=m} C(l,m) b_l(parent) s^(l-m). */
void fo_l2l(int nlevels, int p, const double* center, double* local) {
    for (int l = 0; l + 1 < nlevels; ++l) {
        int64_t off = level_offset(l), nb = fo_num_boxes(l + 1) - off;
#pragma omp parallel for schedule(static)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t g = off + b;
            cplx cp = center[2 * g] + I * center[2 * g + 1];
            for (int c = 0; c < 4; ++c) {
                int64_t h = level_offset(l + 1) + 4 * b + c;
                cplx s = (center[2 * h] + I * center[2 * h + 1]) - cp;
                for (int m = 0; m < p; ++m) {
                    cplx acc = 0;
                    for (int q = m; q < p; ++q) acc += binom(q, m) * load_c(local, g * p + q) * cpow_int(s, q - m);
                    store_c(local, h * p + m, load_c(local, h * p + m) + acc);
                }
            }
        }
    }
}

/* L2P at every point of every leaf; phi/dphi indexed by ORIGINAL point index. */
void fo_l2p(int nlevels, int p, const double* xy, const int64_t* perm, const int64_t* bstart, const int64_t* bcount,
            const double* center, const double* local, double* phi, double* dphi) {
    int64_t l0 = level_offset(nlevels - 1), nb = fo_num_boxes(nlevels) - l0;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t g = l0 + b;
        cplx c = center[2 * g] + I * center[2 * g + 1];
        for (int64_t i = bstart[g]; i < bstart[g] + bcount[g]; ++i) {
            int64_t j = perm[i];
            cplx w = (xy[2 * j] + I * xy[2 * j + 1]) - c;
            cplx v = 0, dv = 0, wl = 1;
            for (int l = 0; l < p; ++l) {
                v += load_c(local, g * p + l) * wl;
                if (l + 1 < p) dv += (double)(l + 1) * load_c(local, g * p + l + 1) * wl;
                wl *= w;
            }
            store_c(phi, j, v);
            if (dphi) store_c(dphi, j, dv);
        }
    }
}

/* P2P: direct sum over the points of the strongly coupled leaves (incl. itself). */
void fo_p2p(int nlevels, const double* xy, const double* gam, const int64_t* perm, const int64_t* bstart,
            const int64_t* bcount, const int64_t* s_off, const int32_t* s_idx, double* phi, double* dphi) {
    int64_t l0 = level_offset(nlevels - 1), nb = fo_num_boxes(nlevels) - l0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t g = l0 + b;
        for (int64_t i = bstart[g]; i < bstart[g] + bcount[g]; ++i) {
            int64_t t = perm[i];
            cplx zt = xy[2 * t] + I * xy[2 * t + 1];
            cplx s = 0, ds = 0;
            for (int64_t q = s_off[g]; q < s_off[g + 1]; ++q) {
                int64_t h = s_idx[q];
                for (int64_t u = bstart[h]; u < bstart[h] + bcount[h]; ++u) {
                    int64_t j = perm[u];
                    cplx zj = xy[2 * j] + I * xy[2 * j + 1];
                    if (zj == zt) continue; /* R7 */
                    cplx r = 1.0 / (zt - zj);
                    s += load_c(gam, j) * r;
                    ds -= load_c(gam, j) * r * r;
                }
            }
            store_c(phi, t, s);
            if (dphi) store_c(dphi, t, ds);
        }
    }
}

/* ------------------------------------------------------------ whole method */

/* One FMM evaluation (Sec. 2.1, Fig 2.2): tree, lists, P2M, M2M, M2L, L2L,
 * L2P, P2P, sum.  Outputs in ORIGINAL point order:
 *   phi  = Phi_near + Phi_far,  dphi = d Phi/dz (optional)
 *   near / far = the two parts (optional);  mpole / local = unscaled
 *   coefficients, nbox*p complex each (optional).
 * Returns 0, -1 on invalid arguments, -2 on allocation failure.             */
int fo_fmm(int64_t n, const double* xy, const double* gam, int nlevels, double theta, int p, double* phi,
           double* dphi, double* mpole_out, double* local_out, double* near_out, double* far_out) {
    if (n < 1 || nlevels < 1 || p < 1 || p > 64 || !(theta > 0.0 && theta < 1.0)) return -1;
    int64_t nbox = fo_num_boxes(nlevels);
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* bstart = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
    int64_t* bcount = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
    double* center = (double*)malloc(sizeof(double) * 2 * (size_t)nbox);
    double* radius = (double*)malloc(sizeof(double) * (size_t)nbox);
    int64_t* s_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    int64_t* w_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    double* mpole = (double*)calloc((size_t)(2 * nbox * p), sizeof(double));
    double* local = (double*)calloc((size_t)(2 * nbox * p), sizeof(double));
    double* nearv = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* farv = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* dnear = dphi ? (double*)malloc(sizeof(double) * 2 * (size_t)n) : NULL;
    double* dfar = dphi ? (double*)malloc(sizeof(double) * 2 * (size_t)n) : NULL;
    int rc = -2;
    if (!perm || !bstart || !bcount || !center || !radius || !s_off || !w_off || !mpole || !local || !nearv ||
        !farv || (dphi && (!dnear || !dfar)))
        goto done;
    rc = fo_build_tree(n, xy, nlevels, perm, bstart, bcount, center, radius);
    if (rc) goto done;
    rc = fo_build_lists(nlevels, center, radius, theta, s_off, w_off, NULL, NULL);
    if (rc) goto done;
    {
        int32_t* s_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s_off[nbox] + 1));
        int32_t* w_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(w_off[nbox] + 1));
        if (!s_idx || !w_idx) { free(s_idx); free(w_idx); rc = -2; goto done; }
        fo_build_lists(nlevels, center, radius, theta, s_off, w_off, s_idx, w_idx);
        fo_p2m(nlevels, p, xy, gam, perm, bstart, bcount, center, mpole);
        fo_m2m(nlevels, p, center, mpole);
        fo_m2l(nlevels, p, center, w_off, w_idx, mpole, local);
        fo_l2l(nlevels, p, center, local);
        fo_l2p(nlevels, p, xy, perm, bstart, bcount, center, local, farv, dfar);
        fo_p2p(nlevels, xy, gam, perm, bstart, bcount, s_off, s_idx, nearv, dnear);
        free(s_idx);
        free(w_idx);
    }
    for (int64_t i = 0; i < 2 * n; ++i) {
        phi[i] = nearv[i] + farv[i];
        if (dphi) dphi[i] = dnear[i] + dfar[i];
        if (near_out) near_out[i] = nearv[i];
        if (far_out) far_out[i] = farv[i];
    }
    if (mpole_out) memcpy(mpole_out, mpole, sizeof(double) * 2 * (size_t)(nbox * p));
    if (local_out) memcpy(local_out, local, sizeof(double) * 2 * (size_t)(nbox * p));
    rc = 0;
done:
    free(perm); free(bstart); free(bcount); free(center); free(radius); free(s_off); free(w_off);
    free(mpole); free(local); free(nearv); free(farv); free(dnear); free(dfar);
    return rc;
}

/* Gradient of L = sum_i w_i Re Phi_i + v_i Im Phi_i (upstream gphi = w + i v)
 * through the FMM with the tree frozen: the adjoint is a second FMM over the
 * same points with strengths c = conj(gphi) giving Psi and Psi', plus Phi'
 * from the forward strengths; the assembly is the one of fo_direct_grad.     */
int fo_fmm_grad(int64_t n, const double* xy, const double* gam, const double* gphi, int nlevels, double theta,
                int p, double* ggam, double* gxy) {
    double* c = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* psi = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* dpsi = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* phi = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* dphi = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    int rc = -2;
    if (!c || !psi || !dpsi || !phi || !dphi) goto done;
    for (int64_t i = 0; i < n; ++i) { c[2 * i] = gphi[2 * i]; c[2 * i + 1] = -gphi[2 * i + 1]; }
    rc = fo_fmm(n, xy, c, nlevels, theta, p, psi, dpsi, NULL, NULL, NULL, NULL);
    if (rc) goto done;
    rc = fo_fmm(n, xy, gam, nlevels, theta, p, phi, dphi, NULL, NULL, NULL, NULL);
    if (rc) goto done;
    for (int64_t k = 0; k < n; ++k) {
        cplx ck = load_c(c, k), D = ck * load_c(dphi, k) - load_c(gam, k) * load_c(dpsi, k);
        store_c(ggam, k, -conj(load_c(psi, k)));
        gxy[2 * k] = creal(D);
        gxy[2 * k + 1] = -cimag(D);
    }
done:
    free(c); free(psi); free(dpsi); free(phi); free(dphi);
    return rc;
}

/* ======================================================= logarithmic kernel
 *
 * The logarithmic potential (Sec. 3.3, used for isopotential plots; its
 * multipole form a_0 log(z - z_0) + sum_j a_j / (z - z_0)^j is the one the paper
 * writes down):
 *     Phi(z_i) = sum_{j: z_j != z_i} Gamma_j ln|z_i - z_j|.
 * Complex strengths act on the real kernel ln|.|, i.e. the real and imaginary
 * parts of Gamma are two real-strength potentials.  For real strengths q,
 * F(z) = sum_j q_j log(z - z_j) has Re F = the potential; the imaginary part of
 * log is branch-dependent and is never used.  Textbook series of the complex
 * log, written out from their definitions:
 *   multipole about c:  F(z) ~ a_0 log(z - c) + sum_{k=1}^{p-1} a_k / (z-c)^k,
 *                       a_0 = sum q_j,  a_k = -sum q_j (z_j - c)^k / k
 *   local about c:      F(z) ~ sum_{l=0}^{p} b_l (z - c)^l
 *   M2M (z0 = c_child - c_parent):
 *       b_0 = a_0,  b_l = -a_0 z0^l / l + sum_{k=1}^{l} a_k z0^(l-k) C(l-1, k-1)
 *   M2L (z0 = c_M - c_L):
 *       b_0 += a_0 log(-z0) + sum_{k>=1} a_k (-1)^k / z0^k
 *       b_l += -a_0 / (l z0^l) + z0^(-l) sum_{k>=1} (a_k / z0^k) C(l+k-1, k-1) (-1)^k
 *   L2L, L2P: Taylor shift and evaluation of the degree-p local polynomial
 *   (fo_l2l / fo_l2p with p+1 coefficients).
 * Truncation: p multipole coefficients (log term + k = 1..p-1) and locals of
 * degree p, so that d/dz of the expansions is the harmonic expansion of p
 * terms used by the rest of this file.                                      */

/* Exact sum at tgt[0..m) (all n points when tgt == NULL). */
void fo_direct_log(int64_t n, const double* xy, const double* gam, int64_t m, const int64_t* tgt, double* phi) {
    if (tgt == NULL) m = n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        int64_t t = tgt ? tgt[q] : q;
        cplx zt = xy[2 * t] + I * xy[2 * t + 1];
        cplx s = 0;
        for (int64_t j = 0; j < n; ++j) {
            cplx zj = xy[2 * j] + I * xy[2 * j + 1];
            if (zj == zt) continue; /* R7 */
            s += load_c(gam, j) * log(cabs(zt - zj));
        }
        store_c(phi, q, s);
    }
}

static void p2m_log(int nlevels, int p, const double* xy, const double* q, const int64_t* perm,
                    const int64_t* bstart, const int64_t* bcount, const double* center, double* mpole) {
    int64_t l0 = level_offset(nlevels - 1), nb = fo_num_boxes(nlevels) - l0;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t g = l0 + b;
        cplx c = center[2 * g] + I * center[2 * g + 1];
        cplx a[64] = {0};
        for (int64_t i = bstart[g]; i < bstart[g] + bcount[g]; ++i) {
            int64_t j = perm[i];
            cplx w = (xy[2 * j] + I * xy[2 * j + 1]) - c;
            a[0] += q[j];
            cplx wk = 1;
            for (int k = 1; k < p; ++k) {
                wk *= w;
                a[k] -= q[j] * wk / (double)k;
            }
        }
        for (int k = 0; k < p; ++k) store_c(mpole, g * p + k, a[k]);
    }
}

static void m2m_log(int nlevels, int p, const double* center, double* mpole) {
    for (int l = nlevels - 2; l >= 0; --l) {
        int64_t off = level_offset(l), nb = fo_num_boxes(l + 1) - off;
#pragma omp parallel for schedule(static)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t g = off + b;
            cplx cp = center[2 * g] + I * center[2 * g + 1];
            cplx out[64] = {0};
            for (int c = 0; c < 4; ++c) {
                int64_t h = level_offset(l + 1) + 4 * b + c;
                cplx z0 = (center[2 * h] + I * center[2 * h + 1]) - cp;
                cplx a0 = load_c(mpole, h * p);
                out[0] += a0;
                for (int n = 1; n < p; ++n) {
                    cplx acc = -a0 * cpow_int(z0, n) / (double)n;
                    for (int k = 1; k <= n; ++k) acc += load_c(mpole, h * p + k) * cpow_int(z0, n - k) * binom(n - 1, k - 1);
                    out[n] += acc;
                }
            }
            for (int n = 0; n < p; ++n) store_c(mpole, g * p + n, out[n]);
        }
    }
}

/* local has p+1 coefficients per box */
static void m2l_log(int nlevels, int p, const double* center, const int64_t* w_off, const int32_t* w_idx,
                    const double* mpole, double* local) {
    int64_t nbox = fo_num_boxes(nlevels);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < nbox; ++g) {
        cplx cl = center[2 * g] + I * center[2 * g + 1];
        cplx b[65] = {0};
        for (int64_t qq = w_off[g]; qq < w_off[g + 1]; ++qq) {
            int64_t h = w_idx[qq];
            cplx z0 = (center[2 * h] + I * center[2 * h + 1]) - cl;
            cplx a0 = load_c(mpole, h * p);
            cplx zi[130]; /* zi[m] = z0^(-m) */
            zi[0] = 1;
            for (int m = 1; m <= 2 * p; ++m) zi[m] = zi[m - 1] / z0;
            cplx b0 = a0 * clog(-z0);
            for (int k = 1; k < p; ++k) b0 += load_c(mpole, h * p + k) * ((k & 1) ? -zi[k] : zi[k]);
            b[0] += b0;
            for (int l = 1; l <= p; ++l) {
                cplx acc = 0;
                for (int k = 1; k < p; ++k) {
                    cplx t = load_c(mpole, h * p + k) * zi[k] * binom(l + k - 1, k - 1);
                    acc += (k & 1) ? -t : t;
                }
                b[l] += -a0 * zi[l] / (double)l + zi[l] * acc;
            }
        }
        for (int l = 0; l <= p; ++l) store_c(local, g * (p + 1) + l, b[l]);
    }
}

static void p2p_log(int nlevels, const double* xy, const double* q, const int64_t* perm, const int64_t* bstart,
                    const int64_t* bcount, const int64_t* s_off, const int32_t* s_idx, double* out) {
    int64_t l0 = level_offset(nlevels - 1), nb = fo_num_boxes(nlevels) - l0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t g = l0 + b;
        for (int64_t i = bstart[g]; i < bstart[g] + bcount[g]; ++i) {
            int64_t t = perm[i];
            cplx zt = xy[2 * t] + I * xy[2 * t + 1];
            double s = 0;
            for (int64_t qq = s_off[g]; qq < s_off[g + 1]; ++qq) {
                int64_t h = s_idx[qq];
                for (int64_t u = bstart[h]; u < bstart[h] + bcount[h]; ++u) {
                    int64_t j = perm[u];
                    cplx zj = xy[2 * j] + I * xy[2 * j + 1];
                    if (zj == zt) continue; /* R7 */
                    s += q[j] * log(cabs(zt - zj));
                }
            }
            out[t] = s;
        }
    }
}

/* One logarithmic-kernel FMM evaluation (complex strengths as two real ones). */
int fo_fmm_log(int64_t n, const double* xy, const double* gam, int nlevels, double theta, int p, double* phi) {
    if (n < 1 || nlevels < 1 || p < 1 || p > 64 || !(theta > 0.0 && theta < 1.0)) return -1;
    int64_t nbox = fo_num_boxes(nlevels);
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* bstart = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
    int64_t* bcount = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
    double* center = (double*)malloc(sizeof(double) * 2 * (size_t)nbox);
    double* radius = (double*)malloc(sizeof(double) * (size_t)nbox);
    int64_t* s_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    int64_t* w_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    double* mpole = (double*)calloc((size_t)(2 * nbox * p), sizeof(double));
    double* local = (double*)calloc((size_t)(2 * nbox * (p + 1)), sizeof(double));
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* nearv = (double*)malloc(sizeof(double) * (size_t)n);
    double* farv = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    int32_t* s_idx = NULL;
    int32_t* w_idx = NULL;
    int rc = -2;
    if (!perm || !bstart || !bcount || !center || !radius || !s_off || !w_off || !mpole || !local || !q || !nearv ||
        !farv)
        goto done;
    rc = fo_build_tree(n, xy, nlevels, perm, bstart, bcount, center, radius);
    if (rc) goto done;
    rc = fo_build_lists(nlevels, center, radius, theta, s_off, w_off, NULL, NULL);
    if (rc) goto done;
    s_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s_off[nbox] + 1));
    w_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(w_off[nbox] + 1));
    if (!s_idx || !w_idx) { rc = -2; goto done; }
    fo_build_lists(nlevels, center, radius, theta, s_off, w_off, s_idx, w_idx);
    for (int part = 0; part < 2; ++part) {  /* real, then imaginary part of the strengths */
        for (int64_t j = 0; j < n; ++j) q[j] = gam[2 * j + part];
        p2m_log(nlevels, p, xy, q, perm, bstart, bcount, center, mpole);
        m2m_log(nlevels, p, center, mpole);
        m2l_log(nlevels, p, center, w_off, w_idx, mpole, local);
        fo_l2l(nlevels, p + 1, center, local);
        fo_l2p(nlevels, p + 1, xy, perm, bstart, bcount, center, local, farv, NULL);
        p2p_log(nlevels, xy, q, perm, bstart, bcount, s_off, s_idx, nearv);
        for (int64_t j = 0; j < n; ++j) phi[2 * j + part] = farv[2 * j] + nearv[j];
    }
    rc = 0;
done:
    free(perm); free(bstart); free(bcount); free(center); free(radius); free(s_off); free(w_off);
    free(mpole); free(local); free(q); free(nearv); free(farv); free(s_idx); free(w_idx);
    return rc;
}
