/*
 * crk_oracle.c -- plain FP64 CPU oracle of the CRKSPH particle-pair passes of
 * CRK-HACC (arXiv 2202.02840, Sec. 1.2 "The CRKSPH Scheme", Sec. 2.6 "Kernel
 * Selection and Smoothing Length").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg and reference arm of bench.py may load this library (the bench
 * times it and, in the CPU baseline leg, states the GPU error against it).
 * It shares no code, header,
 * table or constant generator with the CUDA path; neither includes the other.
 *
 * Everything is FP64 and written literally from the paper's equations, one
 * term per line, with a brute-force O(N^2) neighbour search (grid level 0) or
 * an equivalent uniform-grid candidate search (grid level > 0) whose candidate
 * lists are sorted by particle index, so both searches give bit-identical sums.
 *
 * Readings where the paper is silent or ambiguous:
 *  R1 neighbour predicate: positions canonicalised to uint32 fixed point
 *     q = floor(s*2^32), minimum image dq = (int32)(q_i - q_j), R^2 = sum dq^2
 *     (exact in uint64); H = floor(h*2^32).  gather(i) = {j : R^2 < H_i^2}
 *     (self included); pair set = {(i,j), i != j : R^2 < max(H_i,H_j)^2}.
 *     The separation handed to the maths is x_ij = dq * 2^-32 (exact in FP64).
 *     The kernel W(r, h_i) is taken as zero unless j is in gather(i).
 *  R2 gradients are taken at fixed h and fixed neighbour volumes V_j.
 *  R3 grad W^R_ji is evaluated with particle j's coefficients, x_ji = -x_ij,
 *     and the gradient with respect to x_j.
 *  R4 grad v is stored [alpha][beta] = d v^alpha / d x^beta.
 *  R5 rho_i = m_i / V_i.
 *  R6 van Leer limiter: phi_VL = 0 when b = 0 or a + b = 0 (r = a/b undefined
 *     or -1); otherwise max(0, min(1, 4r/(1+r)^2)).
 *  R7 Q_j of a pair uses j's own h_hat, c_s, rho with the same u_hat_ij.x_ij.
 *  R8 direct energy equation uses P + Q for P_j.
 *  R9 signal velocity v_sig,i = max_j max(0, -(v_i - v_j).x_ij / |x_ij|)
 *     over the pair set (zero for coincident particles).
 * R10 compatible energy: Delta E_ij = 1/2 (v_j + v'_j - v_i - v'_i).F_ij,
 *     f_ij = 1/2 when s_i + s_j = 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

static const double ORC_PI = 3.14159265358979323846;
static const double TWO32 = 4294967296.0;

/* parameter vector layout (double prm[]) */
enum { P_GAMMA = 0, P_NH, P_NRES, P_CL, P_CQ, P_EPS, P_ETACRIT, P_ETAFOLD,
       P_CCFL, P_ZETA, P_A, P_ADOT, P_COUNT };

/* ---------------------------------------------------------------- system */

typedef struct {
    int n, k, nc;          /* grid level k (0 = brute force), nc = 2^k cells/axis */
    uint32_t *q;           /* 3n fixed-point coordinates (R1) */
    uint32_t *H;           /* n fixed-point smoothing lengths (R1) */
    double *h;             /* n smoothing lengths */
    int *cstart, *cidx;    /* grid: particles of cell c are cidx[cstart[c] .. cstart[c+1]) */
    uint32_t *cHmax;       /* grid: max H in each cell */
} sys_t;

static void sys_free(sys_t *s) {
    free(s->q); free(s->H); free(s->h); free(s->cstart); free(s->cidx); free(s->cHmax);
    memset(s, 0, sizeof(*s));
}

static inline int cell_of(const sys_t *s, int i) {
    int sh = 32 - s->k;
    uint32_t cx = s->q[3 * i] >> sh, cy = s->q[3 * i + 1] >> sh, cz = s->q[3 * i + 2] >> sh;
    return (int)((cz * (uint32_t)s->nc + cy) * (uint32_t)s->nc + cx);
}

/* pos4 = n records (x, y, z, h), FP32, x,y,z in [0,1), 0 < h < 1/3. */
static int sys_init(sys_t *s, int n, const float *pos4, int k) {
    memset(s, 0, sizeof(*s));
    if (n < 0 || k < 0 || k > 9) return ORC_EINVAL;
    s->n = n; s->k = k; s->nc = 1 << k;
    s->q = malloc(sizeof(uint32_t) * 3 * (size_t)(n ? n : 1));
    s->H = malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    s->h = malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!s->q || !s->H || !s->h) { sys_free(s); return ORC_ENOMEM; }
    for (int i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) {
            double c = (double)pos4[4 * i + a];
            if (!(c >= 0.0 && c < 1.0)) { sys_free(s); return ORC_EINVAL; }
            s->q[3 * i + a] = (uint32_t)floor(c * TWO32);
        }
        double h = (double)pos4[4 * i + 3];
        if (!(h > 0.0 && h < 1.0 / 3.0)) { sys_free(s); return ORC_EINVAL; }
        s->h[i] = h;
        s->H[i] = (uint32_t)floor(h * TWO32);
    }
    if (k > 0) {
        int ncell = s->nc * s->nc * s->nc;
        s->cstart = calloc((size_t)ncell + 1, sizeof(int));
        s->cidx = malloc(sizeof(int) * (size_t)(n ? n : 1));
        s->cHmax = calloc((size_t)ncell, sizeof(uint32_t));
        if (!s->cstart || !s->cidx || !s->cHmax) { sys_free(s); return ORC_ENOMEM; }
        for (int i = 0; i < n; i++) {
            int c = cell_of(s, i);
            s->cstart[c + 1]++;
            if (s->H[i] > s->cHmax[c]) s->cHmax[c] = s->H[i];
        }
        for (int c = 0; c < ncell; c++) s->cstart[c + 1] += s->cstart[c];
        int *fill = malloc(sizeof(int) * (size_t)ncell);
        if (!fill) { sys_free(s); return ORC_ENOMEM; }
        memcpy(fill, s->cstart, sizeof(int) * (size_t)ncell);
        for (int i = 0; i < n; i++) s->cidx[fill[cell_of(s, i)]++] = i;
        free(fill);
    }
    return ORC_OK;
}

/* ------------------------------------------------------ pair geometry (R1) */

static inline int64_t min_image(uint32_t a, uint32_t b) { return (int64_t)(int32_t)(a - b); }

/* R^2 in fixed point (exact) and x_ij in FP64 box units. */
static inline uint64_t pair_sep(const sys_t *s, int i, int j, double x[3]) {
    uint64_t R2 = 0;
    for (int a = 0; a < 3; a++) {
        int64_t d = min_image(s->q[3 * i + a], s->q[3 * j + a]);
        R2 += (uint64_t)(d * d);
        x[a] = ldexp((double)d, -32);
    }
    return R2;
}

static inline int in_gather(const sys_t *s, int i, uint64_t R2) {
    return R2 < (uint64_t)s->H[i] * (uint64_t)s->H[i];
}

/* ------------------------------------------------------ neighbour search */

typedef struct { int *v; int n, cap; } ilist;

static int ilist_push(ilist *l, int j) {
    if (l->n == l->cap) {
        int nc = l->cap ? 2 * l->cap : 1024;
        int *nv = realloc(l->v, sizeof(int) * (size_t)nc);
        if (!nv) return ORC_ENOMEM;
        l->v = nv; l->cap = nc;
    }
    l->v[l->n++] = j;
    return ORC_OK;
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

enum { MODE_GATHER = 0, MODE_UNION = 1 };

static inline int pair_pred(const sys_t *s, int i, int j, int mode) {
    double x[3];
    uint64_t R2 = pair_sep(s, i, j, x);
    if (mode == MODE_GATHER) return in_gather(s, i, R2);
    if (i == j) return 0;
    uint64_t Hm = s->H[i] > s->H[j] ? s->H[i] : s->H[j];
    return R2 < Hm * Hm;
}

/* Circular distance (fixed point) from coordinate q to the cell interval
 * [lo, lo + w - 1] on the periodic axis of length 2^32. */
static inline uint64_t cell_gap(uint32_t q, uint32_t lo, uint32_t w) {
    uint32_t hi = lo + (w - 1u);
    if (q >= lo && q <= hi) return 0;
    uint32_t d1 = lo - q, d2 = q - hi;   /* both wrap modulo 2^32 */
    return d1 < d2 ? d1 : d2;
}

/* All j in gather(i) (mode 0) or the pair set of i (mode 1), ascending j. */
static int neighbours(const sys_t *s, int i, int mode, uint32_t Hmax_all, ilist *out) {
    out->n = 0;
    if (s->k == 0) {
        for (int j = 0; j < s->n; j++)
            if (pair_pred(s, i, j, mode) && ilist_push(out, j)) return ORC_ENOMEM;
        return ORC_OK;
    }
    uint32_t sh = (uint32_t)(32 - s->k), w = (uint32_t)(1ull << sh) ;
    uint64_t R = (mode == MODE_GATHER) ? s->H[i] : (s->H[i] > Hmax_all ? s->H[i] : Hmax_all);
    int64_t m = (int64_t)(R >> sh) + 1;
    int nc = s->nc, full = (2 * m + 1 >= nc);
    int ci[3];
    for (int a = 0; a < 3; a++) ci[a] = (int)(s->q[3 * i + a] >> sh);
    int lo = full ? 0 : (int)-m, hi = full ? nc - 1 : (int)m;
    for (int dz = lo; dz <= hi; dz++) {
        int cz = full ? dz : ((ci[2] + dz) % nc + nc) % nc;
        uint64_t gz = cell_gap(s->q[3 * i + 2], (uint32_t)cz << sh, w);
        for (int dy = lo; dy <= hi; dy++) {
            int cy = full ? dy : ((ci[1] + dy) % nc + nc) % nc;
            uint64_t gy = cell_gap(s->q[3 * i + 1], (uint32_t)cy << sh, w);
            for (int dx = lo; dx <= hi; dx++) {
                int cx = full ? dx : ((ci[0] + dx) % nc + nc) % nc;
                uint64_t gx = cell_gap(s->q[3 * i], (uint32_t)cx << sh, w);
                int c = (cz * nc + cy) * nc + cx;
                uint64_t g2 = gx * gx + gy * gy + gz * gz;
                uint64_t Rc = R;
                if (mode == MODE_UNION) Rc = s->H[i] > s->cHmax[c] ? s->H[i] : s->cHmax[c];
                if (g2 >= Rc * Rc) continue;
                for (int t = s->cstart[c]; t < s->cstart[c + 1]; t++) {
                    int j = s->cidx[t];
                    if (pair_pred(s, i, j, mode) && ilist_push(out, j)) return ORC_ENOMEM;
                }
            }
        }
    }
    qsort(out->v, (size_t)out->n, sizeof(int), cmp_int);
    return ORC_OK;
}

static uint32_t sys_Hmax(const sys_t *s) {
    uint32_t m = 0;
    for (int i = 0; i < s->n; i++) if (s->H[i] > m) m = s->H[i];
    return m;
}

/* ------------------------------------------------------------- kernel */

/* C4 Wendland kernel, eq:C4: W = 495/(32 pi h^3) (1-eta)^6 (1 + 6 eta + 35/3 eta^2). */
static double W_c4(double r, double h) {
    double eta = r / h;
    if (eta >= 1.0) return 0.0;
    double t = 1.0 - eta;
    return 495.0 / (32.0 * ORC_PI * h * h * h) * pow(t, 6) * (1.0 + 6.0 * eta + 35.0 / 3.0 * eta * eta);
}

/* Gradient of eq:C4 with respect to x_i at fixed h (R2):
 *   dW/deta = -1155/(4 pi h^3) eta (1 + 5 eta) (1 - eta)^5,
 *   grad_i W = (dW/deta) (1/h) x_ij / r = -1155/(4 pi h^5) (1 + 5 eta)(1 - eta)^5 x_ij. */
static void gradW_c4(const double x[3], double r, double h, double g[3]) {
    double eta = r / h;
    if (eta >= 1.0) { g[0] = g[1] = g[2] = 0.0; return; }
    double c = -1155.0 / (4.0 * ORC_PI * pow(h, 5)) * (1.0 + 5.0 * eta) * pow(1.0 - eta, 5);
    for (int a = 0; a < 3; a++) g[a] = c * x[a];
}

/* Kernel value and gradient of the pair (i,j) with i's smoothing length, gated
 * by the fixed-point support predicate (R1). */
static void kern_i(const sys_t *s, int i, uint64_t R2, const double x[3], double r, double *w, double g[3]) {
    if (in_gather(s, i, R2)) { *w = W_c4(r, s->h[i]); gradW_c4(x, r, s->h[i], g); }
    else { *w = 0.0; g[0] = g[1] = g[2] = 0.0; }
}

static inline double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* eq:gRK: grad W^R = grad A (1 + B.x) W + A (grad B . x + B) W + A (1 + B.x) grad W,
 * with gB stored [alpha][gamma] = d B^alpha / d x^gamma. */
static void grad_rk(double A, const double B[3], const double gA[3], const double gB[9],
                    const double x[3], double w, const double gw[3], double out[3]) {
    double s = 1.0 + dot3(B, x);
    for (int g = 0; g < 3; g++) {
        double gBx = 0.0;
        for (int a = 0; a < 3; a++) gBx += gB[3 * a + g] * x[a];
        out[g] = gA[g] * s * w + A * (gBx + B[g]) * w + A * s * gw[g];
    }
}

/* ---------------------------------------------------------- target loop */

static int *make_targets(int n, const int *tgt, int ntgt, int *nt_out) {
    int *t = malloc(sizeof(int) * (size_t)((tgt ? ntgt : n) + 1));
    if (!t) return NULL;
    if (tgt) { for (int k = 0; k < ntgt; k++) t[k] = tgt[k]; *nt_out = ntgt; }
    else { for (int k = 0; k < n; k++) t[k] = k; *nt_out = n; }
    return t;
}

static int check_targets(int n, const int *t, int nt) {
    for (int k = 0; k < nt; k++) if (t[k] < 0 || t[k] >= n) return ORC_EINVAL;
    return ORC_OK;
}

/* ====================================================== exported passes */

/* Fixed-point canonical coordinates (R1): q (3n) and H (n). */
int orc_fixed_point(int n, const float *pos4, uint32_t *q, uint32_t *H) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, 0);
    if (rc) return rc;
    memcpy(q, s.q, sizeof(uint32_t) * 3 * (size_t)n);
    memcpy(H, s.H, sizeof(uint32_t) * (size_t)n);
    sys_free(&s);
    return ORC_OK;
}

/* Neighbour sets.  mode 0: gather(i) incl. i; mode 1: pair set of i.
 * counts[k] = |set(t_k)|.  If lists != NULL it receives the concatenated,
 * ascending lists in target order (capacity cap entries). */
int orc_neighbours(int n, const float *pos4, int k, int mode, const int *tgt, int ntgt,
                   int *counts, int *lists, long long cap) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    uint32_t Hm = sys_Hmax(&s);
    int err = 0;
#pragma omp parallel
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            if (neighbours(&s, t[kk], mode, Hm, &l)) { err = ORC_ENOMEM; continue; }
            counts[kk] = l.n;
        }
        free(l.v);
    }
    if (!err && lists) {
        long long off = 0;
        ilist l = {0};
        for (int kk = 0; kk < nt && !err; kk++) {
            if (neighbours(&s, t[kk], mode, Hm, &l)) { err = ORC_ENOMEM; break; }
            if (off + l.n > cap) { err = ORC_EINVAL; break; }
            memcpy(lists + off, l.v, sizeof(int) * (size_t)l.n);
            off += l.n;
        }
        free(l.v);
    }
    free(t);
    sys_free(&s);
    return err;
}

/* Chaining-mesh binning (reading of the cell list, Sec. 2.3 / D1):
 *  - key = 30-bit Morton interleave of the top 10 bits of (qx, qy, qz), x in bit 0;
 *  - perm = stable sort of particle indices by key (ties by index);
 *  - level k = largest k with 2^-k >= max_i h_i, clamped to [1, kmax];
 *  - cell of a particle = key >> (30 - 3k); cell_start[c] = first sorted
 *    position with cell >= c, for c = 0 .. 8^k (so cell_start[8^k] = n). */
typedef struct { uint32_t key; int idx; } kv_t;
static int cmp_kv(const void *a, const void *b) {
    const kv_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

int orc_cells(int n, const float *pos4, int kmax, uint32_t *key, int *perm, int *k_out, int *cell_start) {
    sys_t s;
    if (n < 0) return ORC_EINVAL;
    int rc = sys_init(&s, n, pos4, 0);
    if (rc) return rc;
    if (kmax < 1 || kmax > 10) { sys_free(&s); return ORC_EINVAL; }
    float hmax = 0.0f;
    for (int i = 0; i < n; i++) if (pos4[4 * i + 3] > hmax) hmax = pos4[4 * i + 3];
    int k = 1;
    if (n > 0) {
        int e;
        double m = frexp((double)hmax, &e);   /* hmax = m 2^e, m in [0.5, 1) */
        k = (m == 0.5) ? 1 - e : -e;
        if (k < 1) k = 1;
        if (k > kmax) k = kmax;
    }
    kv_t *kv = malloc(sizeof(kv_t) * (size_t)(n ? n : 1));
    if (!kv) { sys_free(&s); return ORC_ENOMEM; }
    for (int i = 0; i < n; i++) {
        uint32_t c[3], kk = 0;
        for (int a = 0; a < 3; a++) c[a] = s.q[3 * i + a] >> 22;
        for (int b = 0; b < 10; b++)
            for (int a = 0; a < 3; a++) kk |= ((c[a] >> b) & 1u) << (3 * b + a);
        key[i] = kk;
        kv[i].key = kk; kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(kv_t), cmp_kv);
    for (int t = 0; t < n; t++) perm[t] = kv[t].idx;
    int ncell = 1 << (3 * k), t = 0;
    for (int c = 0; c <= ncell; c++) {
        while (t < n && (int)(kv[t].key >> (30 - 3 * k)) < c) t++;
        cell_start[c] = t;
    }
    *k_out = k;
    free(kv);
    sys_free(&s);
    return ORC_OK;
}

/* P1 -- eq:vol and eq:hi: n_i = sum_{j in gather(i)} W(|x_ij|, h_i), V_i = 1/n_i,
 * N_i = 4/3 pi h_i^3 n_i.  npairs = sum_i (|gather(i)| - 1). */
int orc_volumes(int n, const float *pos4, int k, const int *tgt, int ntgt,
                double *nsum, double *V, double *Nngb, long long *npairs) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    uint32_t Hm = sys_Hmax(&s);
    long long pairs = 0;
    int err = 0;
#pragma omp parallel reduction(+ : pairs)
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            int i = t[kk];
            if (neighbours(&s, i, MODE_GATHER, Hm, &l)) { err = ORC_ENOMEM; continue; }
            double sum = 0.0;
            for (int m = 0; m < l.n; m++) {
                int j = l.v[m];
                double x[3];
                pair_sep(&s, i, j, x);
                sum += W_c4(sqrt(dot3(x, x)), s.h[i]);
            }
            nsum[i] = sum;
            V[i] = 1.0 / sum;
            Nngb[i] = 4.0 / 3.0 * ORC_PI * s.h[i] * s.h[i] * s.h[i] * sum;
            pairs += l.n - 1;
        }
        free(l.v);
    }
    if (npairs) *npairs = pairs;
    free(t);
    sys_free(&s);
    return err;
}

/* Inverse of a 3x3 matrix by adjugate / determinant (row-major). Returns det. */
static double inv3(const double m[9], double inv[9]) {
    double c00 = m[4] * m[8] - m[5] * m[7];
    double c01 = m[5] * m[6] - m[3] * m[8];
    double c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    inv[0] = c00 / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
    return det;
}

static double norm1_3(const double m[9]) {
    double best = 0.0;
    for (int c = 0; c < 3; c++) {
        double s = fabs(m[c]) + fabs(m[3 + c]) + fabs(m[6 + c]);
        if (s > best) best = s;
    }
    return best;
}

/* P2 -- moments over gather(i) and the RK coefficients of eq:RK / eq:gRK, from
 * the two moment conditions sum_j V_j W^R_ij = 1 and sum_j V_j x_ij W^R_ij = 0:
 *   m0 = sum V_j W_ij,  m1^a = sum V_j x^a W_ij,  m2^ab = sum V_j x^a x^b W_ij,
 *   d_g m0 = sum V_j d_g W_ij,
 *   d_g m1^a = sum V_j (delta_ag W_ij + x^a d_g W_ij),
 *   d_g m2^ab = sum V_j (delta_ag x^b W_ij + x^a delta_bg W_ij + x^a x^b d_g W_ij),
 *   B = -m2^-1 m1,  A = 1 / (m0 + m1.B),
 *   d_g B = -m2^-1 (d_g m1 + (d_g m2) B),
 *   d_g A = -A^2 (d_g m0 + B.d_g m1 + m1.d_g B).
 * Outputs: A (n), B (3n), gA (3n, [gamma]), gB (9n, [alpha][gamma]),
 * optional mom (40n: m0, m1[3], m2 {xx,xy,xz,yy,yz,zz}, dm0[3], dm1[a][g] (9),
 * dm2 {xx,xy,xz,yy,yz,zz}[g] (18)), cond (n, 1-norm condition of m2) and
 * optional scale (16n: A, B[3], gA[3], gB[9]) -- the no-cancellation magnitude
 * of each coefficient: the same formulas applied to the absolute values of the
 * pair terms (|x| for x, |W'| for the kernel gradient) and of the factors they
 * multiply, i.e. the first-order bound on how far a rounding of the pair terms
 * can move the coefficient. */
int orc_corrections(int n, const float *pos4, int k, const int *tgt, int ntgt, const double *V,
                    double *A, double *B, double *gA, double *gB, double *mom, double *cond,
                    double *scale) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    uint32_t Hm = sys_Hmax(&s);
    int err = 0;
#pragma omp parallel
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            int i = t[kk];
            if (neighbours(&s, i, MODE_GATHER, Hm, &l)) { err = ORC_ENOMEM; continue; }
            double m0 = 0, m1[3] = {0}, m2[9] = {0}, dm0[3] = {0}, dm1[9] = {0}, dm2[27] = {0};
            double a1[3] = {0}, ad0[3] = {0}, ad1[9] = {0}, ad2[27] = {0};   /* |term| sums */
            for (int m = 0; m < l.n; m++) {
                int j = l.v[m];
                double x[3], gw[3];
                pair_sep(&s, i, j, x);
                double r = sqrt(dot3(x, x));
                double w = W_c4(r, s.h[i]);
                gradW_c4(x, r, s.h[i], gw);
                double Vj = V[j];
                m0 += Vj * w;
                for (int a = 0; a < 3; a++) {
                    m1[a] += Vj * x[a] * w;
                    dm0[a] += Vj * gw[a];
                    for (int b = 0; b < 3; b++) m2[3 * a + b] += Vj * x[a] * x[b] * w;
                    a1[a] += Vj * fabs(x[a]) * w;
                    ad0[a] += Vj * fabs(gw[a]);
                    for (int g = 0; g < 3; g++) {
                        double dag = (a == g) ? 1.0 : 0.0;
                        dm1[3 * a + g] += Vj * (dag * w + x[a] * gw[g]);
                        ad1[3 * a + g] += Vj * (dag * w + fabs(x[a] * gw[g]));
                        for (int b = 0; b < 3; b++) {
                            double dbg = (b == g) ? 1.0 : 0.0;
                            dm2[9 * a + 3 * b + g] += Vj * (dag * x[b] * w + x[a] * dbg * w + x[a] * x[b] * gw[g]);
                            ad2[9 * a + 3 * b + g] += Vj * (dag * fabs(x[b]) * w + fabs(x[a]) * dbg * w +
                                                             fabs(x[a] * x[b] * gw[g]));
                        }
                    }
                }
            }
            double mi[9];
            inv3(m2, mi);
            double Bi[3], Ai, dB[9], dA[3];
            for (int a = 0; a < 3; a++) Bi[a] = -(mi[3 * a] * m1[0] + mi[3 * a + 1] * m1[1] + mi[3 * a + 2] * m1[2]);
            Ai = 1.0 / (m0 + dot3(m1, Bi));
            for (int g = 0; g < 3; g++) {
                double rhs[3];
                for (int a = 0; a < 3; a++) {
                    rhs[a] = dm1[3 * a + g];
                    for (int b = 0; b < 3; b++) rhs[a] += dm2[9 * a + 3 * b + g] * Bi[b];
                }
                for (int a = 0; a < 3; a++)
                    dB[3 * a + g] = -(mi[3 * a] * rhs[0] + mi[3 * a + 1] * rhs[1] + mi[3 * a + 2] * rhs[2]);
            }
            for (int g = 0; g < 3; g++) {
                double acc = dm0[g];
                for (int a = 0; a < 3; a++) acc += Bi[a] * dm1[3 * a + g] + m1[a] * dB[3 * a + g];
                dA[g] = -Ai * Ai * acc;
            }
            A[i] = Ai;
            for (int a = 0; a < 3; a++) { B[3 * i + a] = Bi[a]; gA[3 * i + a] = dA[a]; }
            for (int e = 0; e < 9; e++) gB[9 * i + e] = dB[e];
            if (cond) cond[i] = norm1_3(m2) * norm1_3(mi);
            if (scale) {
                double mia[9], sB[3], sdB[9], sdA[3];
                for (int e = 0; e < 9; e++) mia[e] = fabs(mi[e]);
                for (int a = 0; a < 3; a++) sB[a] = mia[3 * a] * a1[0] + mia[3 * a + 1] * a1[1] + mia[3 * a + 2] * a1[2];
                for (int g = 0; g < 3; g++) {
                    double r[3];
                    for (int a = 0; a < 3; a++) {
                        r[a] = ad1[3 * a + g];
                        for (int b = 0; b < 3; b++) r[a] += ad2[9 * a + 3 * b + g] * fabs(Bi[b]);
                    }
                    for (int a = 0; a < 3; a++) sdB[3 * a + g] = mia[3 * a] * r[0] + mia[3 * a + 1] * r[1] + mia[3 * a + 2] * r[2];
                }
                for (int g = 0; g < 3; g++) {
                    double acc = ad0[g];
                    for (int a = 0; a < 3; a++)
                        acc += fabs(Bi[a]) * ad1[3 * a + g] + a1[a] * fabs(dB[3 * a + g]) + fabs(m1[a]) * sdB[3 * a + g];
                    sdA[g] = Ai * Ai * acc;
                }
                double *o = scale + 16 * (size_t)i;
                o[0] = fabs(Ai);
                for (int a = 0; a < 3; a++) { o[1 + a] = sB[a]; o[4 + a] = sdA[a]; }
                for (int e = 0; e < 9; e++) o[7 + e] = sdB[e];
            }
            if (mom) {
                static const int sa[6] = {0, 0, 0, 1, 1, 2}, sb[6] = {0, 1, 2, 1, 2, 2};
                double *o = mom + 40 * (size_t)i;
                o[0] = m0;
                for (int a = 0; a < 3; a++) o[1 + a] = m1[a];
                for (int p = 0; p < 6; p++) o[4 + p] = m2[3 * sa[p] + sb[p]];
                for (int g = 0; g < 3; g++) o[10 + g] = dm0[g];
                for (int e = 0; e < 9; e++) o[13 + e] = dm1[e];
                for (int p = 0; p < 6; p++)
                    for (int g = 0; g < 3; g++) o[22 + 3 * p + g] = dm2[9 * sa[p] + 3 * sb[p] + g];
            }
        }
        free(l.v);
    }
    free(t);
    sys_free(&s);
    return err;
}

/* P3 -- eq:gradv: grad v_i = - sum_{j in gather(i)} V_j (v_i - v_j) (x) grad W^R_ij,
 * stored [alpha][beta] = d v^alpha / d x^beta (R4).  vel is 3n FP64. */
int orc_gradv(int n, const float *pos4, int k, const int *tgt, int ntgt, const double *V,
              const double *vel, const double *A, const double *B, const double *gA,
              const double *gB, double *gv) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    uint32_t Hm = sys_Hmax(&s);
    int err = 0;
#pragma omp parallel
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            int i = t[kk];
            if (neighbours(&s, i, MODE_GATHER, Hm, &l)) { err = ORC_ENOMEM; continue; }
            double acc[9] = {0};
            for (int m = 0; m < l.n; m++) {
                int j = l.v[m];
                double x[3], gw[3], grk[3];
                pair_sep(&s, i, j, x);
                double r = sqrt(dot3(x, x));
                double w = W_c4(r, s.h[i]);
                gradW_c4(x, r, s.h[i], gw);
                grad_rk(A[i], B + 3 * i, gA + 3 * i, gB + 9 * i, x, w, gw, grk);
                for (int a = 0; a < 3; a++) {
                    double dv = vel[3 * i + a] - vel[3 * j + a];
                    for (int b = 0; b < 3; b++) acc[3 * a + b] += -V[j] * dv * grk[b];
                }
            }
            for (int e = 0; e < 9; e++) gv[9 * i + e] = acc[e];
        }
        free(l.v);
    }
    free(t);
    sys_free(&s);
    return err;
}

/* Per-particle state shared by P4 and P5. */
typedef struct {
    const double *prm, *V, *mass, *vel, *u, *A, *B, *gA, *gB, *gv;
    const double *rho;   /* density of each particle (R5: m / V when NULL) */
} fstate_t;

static double dens(const fstate_t *f, int i) { return f->rho ? f->rho[i] : f->mass[i] / f->V[i]; }

/* eq:phiVL / eq:rij with reading R6 */
static double phi_vanleer(double a, double b) {
    if (b == 0.0 || a + b == 0.0) return 0.0;
    double r = a / b;
    double f = 4.0 * r / ((1.0 + r) * (1.0 + r));
    return f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
}

/* Pairwise quantities of one (i,j) in the pair set, eq:mom, eq:eng, eq:visc,
 * eq:mu, eq:hatvi, eq:phi..eq:phiad, in comoving variables with scale factor a
 * and its rate adot (prm[P_A], prm[P_ADOT]): vel holds p = a^2 dx/dt = a v, gv
 * the gradient of the peculiar velocity v = p / a.
 * F = m_i dp_ij/dt = a^2/2 V_i V_j (P~_i + P~_j)(grad W^R_ji - grad W^R_ij);
 * u^_ij = (p_i - p_j)/a - 1/2 phi (grad v_i + grad v_j).x_ij + adot x_ij (the
 * projection acts on the peculiar part only), mu_i = min(0, (h^_i/a) u^.x /
 * (r^2 + h^_i^2 eps^2)); the approach speed of the signal velocity takes
 * dx/dt_ij + (adot/a) x_ij.  Also returns D = grad W^R_ji - grad W^R_ij, P~_j
 * and Q_i of this pair. */
static void pair_force(const sys_t *s, const fstate_t *f, int i, int j,
                       double F[3], double D[3], double *Ptj, double *Qi_out, double *xr_out) {
    const double *prm = f->prm;
    double gam = prm[P_GAMMA];
    double x[3], xj[3], wi, wj, gwi[3], gwj[3], gri[3], grj[3];
    uint64_t R2 = pair_sep(s, i, j, x);
    double r = sqrt(dot3(x, x));
    for (int a = 0; a < 3; a++) xj[a] = -x[a];
    kern_i(s, i, R2, x, r, &wi, gwi);
    kern_i(s, j, R2, xj, r, &wj, gwj);
    grad_rk(f->A[i], f->B + 3 * i, f->gA + 3 * i, f->gB + 9 * i, x, wi, gwi, gri);
    grad_rk(f->A[j], f->B + 3 * j, f->gA + 3 * j, f->gB + 9 * j, xj, wj, gwj, grj);
    for (int a = 0; a < 3; a++) D[a] = grj[a] - gri[a];

    /* thermodynamics, eq:EOS with rho = m / V (R5) */
    double rho_i = dens(f, i), rho_j = dens(f, j);
    double P_i = (gam - 1.0) * rho_i * f->u[i], P_j = (gam - 1.0) * rho_j * f->u[j];
    double c_i = sqrt(gam * P_i / rho_i), c_j = sqrt(gam * P_j / rho_j);

    /* limiter, eq:phi .. eq:phiad */
    const double *Gi = f->gv + 9 * i, *Gj = f->gv + 9 * j;
    double qa = 0.0, qb = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) { qa += x[a] * Gi[3 * a + b] * x[b]; qb += x[a] * Gj[3 * a + b] * x[b]; }
    double phiVL = phi_vanleer(qa, qb);
    double eta_i = r / s->h[i], eta_j = r / s->h[j];
    double eta = eta_i < eta_j ? eta_i : eta_j;
    double ec = prm[P_ETACRIT], ef = prm[P_ETAFOLD];
    double phiad = (eta < ec) ? exp(-((eta - ec) / ef) * ((eta - ec) / ef)) : 1.0;
    double phi = phiVL * phiad;

    /* midpoint-projected proper velocity difference, eq:hatvi */
    const double sa = prm[P_A], sadot = prm[P_ADOT];
    double uh[3];
    for (int a = 0; a < 3; a++) {
        double proj = 0.0;
        for (int b = 0; b < 3; b++) proj += (Gi[3 * a + b] + Gj[3 * a + b]) * x[b];
        uh[a] = (f->vel[3 * i + a] - f->vel[3 * j + a]) / sa - 0.5 * phi * proj + sadot * x[a];
    }
    double ux = dot3(uh, x);

    /* viscosity, eq:visc / eq:mu with R7 */
    double eps = prm[P_EPS], Cl = prm[P_CL], Cq = prm[P_CQ], nh = prm[P_NH];
    double hh_i = s->h[i] / nh, hh_j = s->h[j] / nh;
    double mu_i = (hh_i / sa) * ux / (r * r + hh_i * hh_i * eps * eps);
    double mu_j = (hh_j / sa) * ux / (r * r + hh_j * hh_j * eps * eps);
    if (mu_i > 0.0) mu_i = 0.0;
    if (mu_j > 0.0) mu_j = 0.0;
    double Q_i = rho_i * (-Cl * c_i * mu_i + Cq * mu_i * mu_i);
    double Q_j = rho_j * (-Cl * c_j * mu_j + Cq * mu_j * mu_j);

    double Pt_i = P_i + Q_i, Pt_j = P_j + Q_j;
    double c = 0.5 * sa * sa * f->V[i] * f->V[j] * (Pt_i + Pt_j);
    for (int a = 0; a < 3; a++) F[a] = c * D[a];
    *Ptj = Pt_j;
    *Qi_out = Q_i;
    /* approach speed for the signal velocity (R9): (dx/dt_ij + (adot/a) x_ij).x_ij / r */
    double vx = 0.0;
    for (int a = 0; a < 3; a++) vx += (f->vel[3 * i + a] - f->vel[3 * j + a]) * x[a];
    vx = vx / (sa * sa) + (sadot / sa) * r * r;
    *xr_out = (r > 0.0 && vx < 0.0) ? -vx / r : 0.0;
}

/* P4 -- eq:mom (momentum), eq:eng (direct energy rate) with P -> P + Q:
 *   acc_i  = dp_i/dt = (1/m_i) sum_j F_ij,
 *   dudt_i = (1/m_i) sum_j 1/(2 a^4) V_i V_j P~_j (p_j - p_i).(grad W^R_ji - grad W^R_ij)
 *            (eq:eng with dx/dt = p / a^2),
 *   vsig_i = max_j approach speed (R9), qmax_i = max_j Q_i of the pair,
 *   fscale_i = (1/m_i) sum_j |F_ij| (scale of the cancelling pair sum, optional). */
int orc_forces(int n, const float *pos4, int k, const int *tgt, int ntgt, const double *prm,
               const double *V, const double *mass, const double *vel, const double *u,
               const double *A, const double *B, const double *gA, const double *gB, const double *gv,
               double *acc, double *dudt, double *vsig, double *qmax, double *fscale,
               long long *npairs, const double *rho) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    fstate_t f = {prm, V, mass, vel, u, A, B, gA, gB, gv, rho};
    uint32_t Hm = sys_Hmax(&s);
    long long pairs = 0;
    int err = 0;
#pragma omp parallel reduction(+ : pairs)
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            int i = t[kk];
            if (neighbours(&s, i, MODE_UNION, Hm, &l)) { err = ORC_ENOMEM; continue; }
            double Fs[3] = {0}, du = 0.0, vs = 0.0, qm = 0.0, fa = 0.0;
            for (int m = 0; m < l.n; m++) {
                int j = l.v[m];
                double F[3], D[3], Ptj, Qi, ap;
                pair_force(&s, &f, i, j, F, D, &Ptj, &Qi, &ap);
                double wdot = 0.0;
                for (int a = 0; a < 3; a++) {
                    Fs[a] += F[a];
                    wdot += (vel[3 * j + a] - vel[3 * i + a]) * D[a];
                }
                fa += sqrt(dot3(F, F));
                du += 0.5 * V[i] * V[j] * Ptj * wdot;
                if (ap > vs) vs = ap;
                if (Qi > qm) qm = Qi;
            }
            const double a4 = prm[P_A] * prm[P_A] * prm[P_A] * prm[P_A];
            for (int a = 0; a < 3; a++) acc[3 * i + a] = Fs[a] / mass[i];
            dudt[i] = du / (a4 * mass[i]);
            vsig[i] = vs;
            if (qmax) qmax[i] = qm;
            if (fscale) fscale[i] = fa / mass[i];
            pairs += l.n;
        }
        free(l.v);
    }
    if (npairs) *npairs = pairs;
    free(t);
    sys_free(&s);
    return err;
}

/* eq:fij with reading R10 */
static double f_partition(double dE, double si, double sj) {
    double sum = si + sj;
    if (sum == 0.0) return 0.5;
    int take_min = (dE >= 0.0 && si >= sj) || (dE < 0.0 && si < sj);
    double lo = si < sj ? si : sj, hi = si < sj ? sj : si;
    return (take_min ? lo : hi) / sum;
}

/* P5 -- compatible energy, eq:compEng2 .. eq:fij:
 *   dp_ij/dt = F_ij / m_i, Delta u_ij = f_ij/(2 a^4) (p_j + p'_j - p_i - p'_i).dp_ij/dt,
 *   Delta E_ij = 1/2 (p_j + p'_j - p_i - p'_i).F_ij (R10), s = P / rho^gamma,
 * with F_ij from the evaluation state (vel, u) and (vb, va) the velocities
 * before and after the kick.  du[i] = sum_j Delta u_ij (multiply by the kick's
 * duration for the energy change). */
int orc_compatible(int n, const float *pos4, int k, const int *tgt, int ntgt, const double *prm,
                   const double *V, const double *mass, const double *vel, const double *u,
                   const double *A, const double *B, const double *gA, const double *gB, const double *gv,
                   const double *vb, const double *va, double *du, const double *rho) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    fstate_t f = {prm, V, mass, vel, u, A, B, gA, gB, gv, rho};
    double gam = prm[P_GAMMA];
    uint32_t Hm = sys_Hmax(&s);
    int err = 0;
#pragma omp parallel
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            int i = t[kk];
            if (neighbours(&s, i, MODE_UNION, Hm, &l)) { err = ORC_ENOMEM; continue; }
            double rho_i = dens(&f, i);
            double s_i = (gam - 1.0) * rho_i * u[i] / pow(rho_i, gam);
            double acc = 0.0;
            for (int m = 0; m < l.n; m++) {
                int j = l.v[m];
                double F[3], D[3], Ptj, Qi, ap;
                pair_force(&s, &f, i, j, F, D, &Ptj, &Qi, &ap);
                double rho_j = dens(&f, j);
                double s_j = (gam - 1.0) * rho_j * u[j] / pow(rho_j, gam);
                double w = 0.0;
                for (int a = 0; a < 3; a++)
                    w += (vb[3 * j + a] + va[3 * j + a] - vb[3 * i + a] - va[3 * i + a]) * F[a];
                double dE = 0.5 * w;
                double fij = f_partition(dE, s_i, s_j);
                acc += fij * 0.5 * w / mass[i];
            }
            du[i] = acc / (prm[P_A] * prm[P_A] * prm[P_A] * prm[P_A]);
        }
        free(l.v);
    }
    free(t);
    sys_free(&s);
    return err;
}

/* RK-corrected density (the density option of crk_params): rho_i = sum over
 * gather(i), self included, of m_j W^R_ij = A_i (1 + B_i . x_ij) W(r_ij, h_i)
 * (eq:RK), the RK interpolant of the field m_j / V_j, which it reproduces when
 * that field is constant or linear. */
int orc_rkdensity(int n, const float *pos4, int k, const int *tgt, int ntgt, const double *mass,
                  const double *A, const double *B, double *rho) {
    sys_t s;
    int rc = sys_init(&s, n, pos4, k);
    if (rc) return rc;
    int nt;
    int *t = make_targets(n, tgt, ntgt, &nt);
    if (!t || check_targets(n, t, nt)) { free(t); sys_free(&s); return t ? ORC_EINVAL : ORC_ENOMEM; }
    uint32_t Hm = sys_Hmax(&s);
    int err = 0;
#pragma omp parallel
    {
        ilist l = {0};
#pragma omp for schedule(dynamic, 16)
        for (int kk = 0; kk < nt; kk++) {
            int i = t[kk];
            if (neighbours(&s, i, MODE_GATHER, Hm, &l)) { err = ORC_ENOMEM; continue; }
            double sum = 0.0;
            for (int m = 0; m < l.n; m++) {
                int j = l.v[m];
                double x[3];
                pair_sep(&s, i, j, x);
                double r = sqrt(dot3(x, x));
                sum += mass[j] * (1.0 + dot3(B + 3 * i, x)) * W_c4(r, s.h[i]);
            }
            rho[i] = A[i] * sum;
        }
        free(l.v);
    }
    free(t);
    sys_free(&s);
    return err;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Kernel values for tests: W[k] = W(r[k], h[k]) (eq:C4) and dWdr[k] = dW/dr. */
int orc_kernel(int n, const double *r, const double *h, double *W, double *dWdr) {
    for (int k = 0; k < n; k++) {
        double x[3] = {r[k], 0.0, 0.0}, g[3];
        W[k] = W_c4(r[k], h[k]);
        gradW_c4(x, r[k], h[k], g);
        dWdr[k] = r[k] > 0.0 ? g[0] : 0.0;   /* grad along +x of a separation (r,0,0) */
    }
    return ORC_OK;
}
