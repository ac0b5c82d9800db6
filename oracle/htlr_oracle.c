/*
 * htlr_oracle.c -- CPU oracle for the hierarchical Tucker low-rank (HTLR) matrix of
 * Li & Liu, "Hierarchical Tucker Low-Rank Matrices: Construction and Matrix-Vector
 * Multiplication" (arXiv 2508.05958).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no code, header,
 * table or constant generator with the CUDA library, and the library never calls it.
 *
 * What it computes (each function cites the passage it follows):
 *   - the Nystrom operator f_i = a(x_i) u_i + sum_j K_ij w_j u_j with the modified
 *     diagonal K_ii w_i = int_{Omega_i} k(x_i, y) dy           (eq. (1.3), (1.4); §3.3)
 *   - Chebyshev points and Lagrange polynomials                 (§3.1)
 *   - the cluster tree by 2^d uniform partition                 (§2.2, Def. 3.3)
 *   - the block cluster tree under weak / strong admissibility  (Def. 2.2, 2.3, 2.4)
 *   - Construct, Algorithm 1: interpolation factors and core (eq. (3.5)), QR of every
 *     factor, core update G <- (w G) x_l R_l x_{d+l} T_l; dense inadmissible leaves
 *     (eq. (4.1))
 *   - HMultVec, Algorithm 2: per-block W = U x_l V_l^T, H = G W, F = H x_l U_l
 *     (eq. (4.3)); dense gemv on inadmissible leaves
 *   - a row-sampled HTLR product and dense product for large N
 *   - the block-tree counts and the paper's storage formula (Prop. 3.4/3.5, Tables 5.1-5.4)
 *
 * Readings where the paper is silent or garbled:
 *   - Lagrange basis: L_t(x) = prod_{j != t} (x - xi_j) / (xi_t - xi_j) (the printed
 *     formula swaps the indices; §3.1).
 *   - Admissibility is tested on the geometric tree cells [k 2^-l, (k+1) 2^-l]^d,
 *     comparing squares: max(diam^2) <= eta^2 dist^2 (1 + 1e-12), so ties are admissible.
 *     eta <= 0 selects weak admissibility: cells with zero-measure overlap.
 *   - Diagonal: Omega_i is split at x_i into 2^d boxes; each gets a q^d Gauss-Legendre
 *     rule, so the singular point is never a node.
 *   - Wide factors (n_box < p): economy QR gives p_eff = min(n_box, p).
 *   - Tensor (non-uniform) grids: the 1-D cell widths are folded into V_l before the
 *     QR; on uniform grids h^d multiplies the core as in Algorithm 1.
 *
 * Layout conventions: natural point order i_1 + n i_2 + n^2 i_3 (first index fastest,
 * §2.1); multi-RHS vectors are N x nrhs column-major; tensors are stored first index
 * fastest; the 2d-order core has the target multi-index t first, source s second.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* Kernel identifiers (same numbering as the library's public enum, so one Python
 * description drives both; the numbers are an interface, not shared code). */
enum { ORC_K_LOG = 0, ORC_K_INV_R = 1, ORC_K_EXP_R = 2, ORC_K_GAUSS = 3,
       ORC_K_POLY = 4, ORC_K_CONST = 5 };

/* ------------------------------------------------------------------------------ */
/* Problem description                                                            */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int d;                 /* dimension, 2 or 3 */
    int n;                 /* points per dimension, N = n^d */
    int ktype;             /* kernel id */
    double kscale;         /* kernel multiplier */
    double kparam;         /* Gaussian sigma, or per-dimension polynomial degree */
    const double *x[3];    /* x[l][i]: coordinate of grid line i in dimension l */
    const double *edge[3]; /* edge[l][i], edge[l][i+1]: cell of grid line i, n+1 values */
    const double *a;       /* a(x_i) in natural order, or NULL for a = 0 */
    int uniform;           /* 1: all cells have width h = 1/n (weight h^d on the core) */
    int q;                 /* Gauss-Legendre order of the diagonal rule */
    int L;                 /* depth of the cluster tree */
    int *bfirst[3];        /* per dimension, per 1-D box of every level (level l at     */
    int *bcnt[3];          /* offset 2^l - 1): first grid line and number of lines      */
} orc_problem;

/* ------------------------------------------------------------------------------ */
/* Kernel functions (§5: Gaussian and SLP kernels; exp(-r); test kernels)           */
/* ------------------------------------------------------------------------------ */
double orc_kernel(const orc_problem *P, const double *x, const double *y)
{
    int d = P->d;
    double r2 = 0.0;
    for (int l = 0; l < d; ++l) {
        double t = x[l] - y[l];
        r2 += t * t;
    }
    switch (P->ktype) {
    case ORC_K_LOG:   return P->kscale * log(sqrt(r2));
    case ORC_K_INV_R: return P->kscale / sqrt(r2);
    case ORC_K_EXP_R: return P->kscale * exp(-sqrt(r2));
    case ORC_K_GAUSS: return P->kscale * exp(-r2 / (2.0 * P->kparam * P->kparam));
    case ORC_K_POLY: {
        /* prod_l (x_l - y_l + 2 + l/2)^deg: degree deg in each coordinate of x and of
         * y, translation invariant, not symmetric in (x, y) nor across dimensions */
        int deg = (int)P->kparam;
        double v = 1.0;
        for (int l = 0; l < d; ++l) {
            double b = x[l] - y[l] + 2.0 + 0.5 * l, pw = 1.0;
            for (int e = 0; e < deg; ++e) pw *= b;
            v *= pw;
        }
        return P->kscale * v;
    }
    case ORC_K_CONST: return P->kscale;
    }
    return NAN;
}

double orc_kernel_eval(int ktype, double kscale, double kparam, int d,
                       const double *x, const double *y)
{
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.d = d; P.ktype = ktype; P.kscale = kscale; P.kparam = kparam;
    return orc_kernel(&P, x, y);
}

/* ------------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1, 1]: Newton's method on the Legendre polynomial P_q,  */
/* evaluated by the three-term recurrence (textbook construction).                  */
/* ------------------------------------------------------------------------------ */
int orc_gauss_legendre(int q, double *node, double *weight)
{
    if (q < 1) return -1;
    for (int i = 0; i < q; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            /* P_q(z) and P_{q-1}(z) by k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2} */
            double pk = z, pkm1 = 1.0;
            for (int k = 2; k <= q; ++k) {
                double pn = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pkm1) / k;
                pkm1 = pk;
                pk = pn;
            }
            /* P_q'(z) = q (z P_q - P_{q-1}) / (z^2 - 1) */
            double dp = q * (z * pk - pkm1) / (z * z - 1.0);
            double dz = pk / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double pk = z, pkm1 = 1.0;
        for (int k = 2; k <= q; ++k) {
            double pn = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pkm1) / k;
            pkm1 = pk;
            pk = pn;
        }
        double dp = q * (z * pk - pkm1) / (z * z - 1.0);
        node[i] = z;
        weight[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* The modified diagonal, eq. (1.4): int_{Omega_i} k(x_i, y) dy.  Omega_i is split    */
/* at x_i into 2^d boxes and each gets a q^d Gauss-Legendre rule.                    */
/* ------------------------------------------------------------------------------ */
double orc_diag_integral(const orc_problem *P, const double *xi, const double *lo,
                         const double *hi)
{
    int d = P->d, q = P->q;
    double *gx = malloc(sizeof(double) * q), *gw = malloc(sizeof(double) * q);
    orc_gauss_legendre(q, gx, gw);
    double total = 0.0;
    for (int c = 0; c < (1 << d); ++c) {
        double a[3], b[3];
        for (int l = 0; l < d; ++l) {
            if ((c >> l) & 1) { a[l] = xi[l]; b[l] = hi[l]; }
            else              { a[l] = lo[l]; b[l] = xi[l]; }
        }
        long npts = 1;
        for (int l = 0; l < d; ++l) npts *= q;
        double s = 0.0;
        for (long m = 0; m < npts; ++m) {
            long r = m;
            double y[3], w = 1.0;
            for (int l = 0; l < d; ++l) {
                int k = (int)(r % q);
                r /= q;
                double half = 0.5 * (b[l] - a[l]);
                y[l] = 0.5 * (a[l] + b[l]) + half * gx[k];
                w *= half * gw[k];
            }
            s += w * orc_kernel(P, xi, y);
        }
        total += s;
    }
    free(gx);
    free(gw);
    return total;
}

double orc_diag_integral_eval(int ktype, double kscale, double kparam, int d, int q,
                              const double *xi, const double *lo, const double *hi)
{
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.d = d; P.ktype = ktype; P.kscale = kscale; P.kparam = kparam; P.q = q;
    return orc_diag_integral(&P, xi, lo, hi);
}

/* ------------------------------------------------------------------------------ */
/* Dense Nystrom product, eq. (1.3)/(1.4) (uniform) and §3.3 (cell measures |Omega_j|) */
/* ------------------------------------------------------------------------------ */
static void point_of(const orc_problem *P, long idx, double *x, int *mi)
{
    for (int l = 0; l < P->d; ++l) {
        int i = (int)(idx % P->n);
        idx /= P->n;
        mi[l] = i;
        x[l] = P->x[l][i];
    }
}

static double cell_measure(const orc_problem *P, const int *mi)
{
    double w = 1.0;
    for (int l = 0; l < P->d; ++l) w *= P->edge[l][mi[l] + 1] - P->edge[l][mi[l]];
    return w;
}

/* f(rows[r], c) for r < nrows and every right-hand side c.  u is N x nrhs
 * column-major; frows is nrows x nrhs column-major. */
int orc_dense_rows(const orc_problem *P, const double *u, int nrhs, const int64_t *rows,
                   int64_t nrows, double *frows)
{
    long N = 1;
    for (int l = 0; l < P->d; ++l) N *= P->n;
    /* cell measures w_j and coordinates, computed once */
    double *w = malloc(sizeof(double) * N);
    double *xs = malloc(sizeof(double) * N * P->d);
    for (long j = 0; j < N; ++j) {
        int mj[3];
        point_of(P, j, xs + j * P->d, mj);
        w[j] = cell_measure(P, mj);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nrows; ++r) {
        long i = (long)rows[r];
        int mi[3];
        double xi[3], lo[3], hi[3];
        point_of(P, i, xi, mi);
        for (int l = 0; l < P->d; ++l) {
            lo[l] = P->edge[l][mi[l]];
            hi[l] = P->edge[l][mi[l] + 1];
        }
        double diag = orc_diag_integral(P, xi, lo, hi) + (P->a ? P->a[i] : 0.0);
        /* one kernel value per pair, used by every right-hand side: the values of a run
         * of columns j are kept, then each right-hand side takes that run; every sum
         * still runs over j in increasing order (j = i contributes through diag) */
        enum { RUN = 4096 };
        double *s = calloc((size_t)nrhs, sizeof(double));
        double *kw = malloc(sizeof(double) * RUN);
        for (long j0 = 0; j0 < N; j0 += RUN) {
            const long j1 = j0 + RUN < N ? j0 + RUN : N;
            for (long j = j0; j < j1; ++j)
                kw[j - j0] = j == i ? 0.0 : orc_kernel(P, xi, xs + j * P->d) * w[j];
            for (int c = 0; c < nrhs; ++c) {
                const double *uc = u + (long)c * N;
                double sc = s[c];
                for (long j = j0; j < j1; ++j)
                    if (j != i) sc += kw[j - j0] * uc[j];
                s[c] = sc;
            }
        }
        for (int c = 0; c < nrhs; ++c)
            frows[r + (long)c * nrows] = s[c] + diag * u[(long)c * N + i];
        free(kw);
        free(s);
    }
    free(w);
    free(xs);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Chebyshev points and Lagrange polynomials on [a, b] (§3.1)                        */
/* ------------------------------------------------------------------------------ */
void orc_cheb_nodes(int p, double a, double b, double *xi)
{
    for (int t = 1; t <= p; ++t)
        xi[t - 1] = 0.5 * (b - a) * cos((2.0 * t - 1.0) * ORC_PI / (2.0 * p)) + 0.5 * (b + a);
}

double orc_lagrange(int p, const double *xi, int t, double x)
{
    double v = 1.0;
    for (int j = 0; j < p; ++j)
        if (j != t) v *= (x - xi[j]) / (xi[t] - xi[j]);
    return v;
}

/* ------------------------------------------------------------------------------ */
/* Householder QR, economy size: A (m x c, column-major) = Q (m x k) R (k x c),      */
/* k = min(m, c).  Used for the orthogonalisation in Algorithm 1 (§2.1).             */
/* ------------------------------------------------------------------------------ */
void orc_qr(int m, int c, const double *A, double *Q, double *R)
{
    int k = m < c ? m : c;
    double *B = malloc(sizeof(double) * m * c);
    double *V = calloc((size_t)m * k, sizeof(double)); /* reflectors v_j, column j */
    double *beta = calloc(k, sizeof(double));
    memcpy(B, A, sizeof(double) * m * c);
    for (int j = 0; j < k; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += B[i + j * m] * B[i + j * m];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = B[j + j * m] >= 0 ? -nrm : nrm;
        double *v = V + (long)j * m;
        for (int i = j; i < m; ++i) v[i] = B[i + j * m];
        v[j] -= alpha;
        double vv = 0.0;
        for (int i = j; i < m; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        beta[j] = 2.0 / vv;
        for (int cc = j; cc < c; ++cc) { /* B <- (I - beta v v^T) B */
            double s = 0.0;
            for (int i = j; i < m; ++i) s += v[i] * B[i + cc * m];
            s *= beta[j];
            for (int i = j; i < m; ++i) B[i + cc * m] -= s * v[i];
        }
    }
    for (int i = 0; i < k; ++i)
        for (int cc = 0; cc < c; ++cc) R[i + cc * k] = (cc >= i) ? B[i + cc * m] : 0.0;
    /* Q = H_0 H_1 ... H_{k-1} [I_k; 0] */
    for (int cc = 0; cc < k; ++cc)
        for (int i = 0; i < m; ++i) Q[i + cc * m] = (i == cc) ? 1.0 : 0.0;
    for (int j = k - 1; j >= 0; --j) {
        if (beta[j] == 0.0) continue;
        const double *v = V + (long)j * m;
        for (int cc = 0; cc < k; ++cc) {
            double s = 0.0;
            for (int i = j; i < m; ++i) s += v[i] * Q[i + cc * m];
            s *= beta[j];
            for (int i = j; i < m; ++i) Q[i + cc * m] -= s * v[i];
        }
    }
    free(B);
    free(V);
    free(beta);
}

/* ------------------------------------------------------------------------------ */
/* Cluster tree (§2.2, Example 2.1, Def. 3.3): the box of level l with multi-index b  */
/* is the cell prod_l [b_l 2^-l, (b_l+1) 2^-l]; it holds the grid lines whose        */
/* coordinate lies in the half-open [b_l 2^-l, (b_l+1) 2^-l) (closed at 1).          */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int level;
    int b[3];      /* box multi-index at its level */
    int first[3];  /* first grid line per dimension */
    int cnt[3];    /* number of grid lines per dimension */
    double lo[3], hi[3];
} orc_box;

/* 1-D membership of every box of every level, by scanning the sorted coordinates. */
static void setup_boxes(orc_problem *P, int L)
{
    P->L = L;
    int nb = (1 << (L + 1)) - 1;
    for (int l = 0; l < P->d; ++l) {
        P->bfirst[l] = malloc(sizeof(int) * nb);
        P->bcnt[l] = malloc(sizeof(int) * nb);
        for (int lev = 0; lev <= L; ++lev) {
            double side = ldexp(1.0, -lev);
            for (int k = 0; k < (1 << lev); ++k) {
                double lo = k * side, hi = (k + 1) * side;
                int first = -1, cnt = 0;
                for (int i = 0; i < P->n; ++i) {
                    double xv = P->x[l][i];
                    int in = (xv >= lo) && (xv < hi || (hi >= 1.0 && xv <= 1.0));
                    if (in) {
                        if (first < 0) first = i;
                        ++cnt;
                    }
                }
                P->bfirst[l][(1 << lev) - 1 + k] = first;
                P->bcnt[l][(1 << lev) - 1 + k] = cnt;
            }
        }
    }
}

static void free_boxes(orc_problem *P)
{
    for (int l = 0; l < 3; ++l) {
        free(P->bfirst[l]);
        free(P->bcnt[l]);
        P->bfirst[l] = P->bcnt[l] = NULL;
    }
}

/* Every node of a cluster tree is non-empty (Def. 2.1). */
static int boxes_nonempty(const orc_problem *P)
{
    int nb = (1 << (P->L + 1)) - 1;
    for (int l = 0; l < P->d; ++l)
        for (int k = 0; k < nb; ++k)
            if (P->bcnt[l][k] < 1) return 0;
    return 1;
}

static void make_box(const orc_problem *P, int level, const int *b, orc_box *B)
{
    B->level = level;
    double side = ldexp(1.0, -level);
    for (int l = 0; l < P->d; ++l) {
        B->b[l] = b[l];
        B->lo[l] = b[l] * side;
        B->hi[l] = (b[l] + 1) * side;
        B->first[l] = P->bfirst[l][(1 << level) - 1 + b[l]];
        B->cnt[l] = P->bcnt[l][(1 << level) - 1 + b[l]];
    }
    for (int l = P->d; l < 3; ++l) {
        B->b[l] = 0; B->first[l] = 0; B->cnt[l] = 1; B->lo[l] = 0; B->hi[l] = 1;
    }
}

/* Admissibility (Def. 2.2 weak, Def. 2.3 strong) on the geometric cells. */
static int admissible(int d, const orc_box *t, const orc_box *s, double eta)
{
    if (eta <= 0.0) {
        /* weak: the two cells overlap in a set of measure zero */
        double vol = 1.0;
        for (int l = 0; l < d; ++l) {
            double lo = t->lo[l] > s->lo[l] ? t->lo[l] : s->lo[l];
            double hi = t->hi[l] < s->hi[l] ? t->hi[l] : s->hi[l];
            double ov = hi - lo;
            vol *= ov > 0 ? ov : 0.0;
        }
        return vol == 0.0;
    }
    double dt = 0, ds = 0, dist = 0;
    for (int l = 0; l < d; ++l) {
        double a = t->hi[l] - t->lo[l], b = s->hi[l] - s->lo[l];
        dt += a * a;
        ds += b * b;
        double g = 0.0;
        if (s->lo[l] > t->hi[l]) g = s->lo[l] - t->hi[l];
        if (t->lo[l] > s->hi[l]) g = t->lo[l] - s->hi[l];
        dist += g * g;
    }
    double diam2 = dt > ds ? dt : ds;
    return diam2 <= eta * eta * dist * (1.0 + 1e-12);
}

/* ------------------------------------------------------------------------------ */
/* Block cluster tree walk (Def. 2.4) and block storage                            */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int far;            /* 1: admissible leaf (TLR block), 0: inadmissible (dense) */
    orc_box tau, sig;
    int pt[3], ps[3];   /* ranks after orthogonalisation, per dimension */
    double *U[3];       /* cnt_tau[l] x pt[l] */
    double *V[3];       /* cnt_sig[l] x ps[l] */
    double *G;          /* prod pt x prod ps (t first) */
    double *D;          /* dense block |tau| x |sigma| (column-major) */
} orc_block;

typedef struct {
    orc_problem P;
    int L, p, orth;
    double eta;
    long nblk, cap;
    orc_block *blk;
    /* owned copies of the problem arrays */
    double *xbuf, *ebuf, *abuf;
} orc_htlr;

void orc_htlr_free(orc_htlr *H);

typedef struct {
    long nblk, cap;
    orc_box *t, *s;
    int *far;
} blist;

static void blist_push(blist *bl, const orc_box *t, const orc_box *s, int far)
{
    if (bl->nblk == bl->cap) {
        bl->cap = bl->cap ? 2 * bl->cap : 1024;
        bl->t = realloc(bl->t, sizeof(orc_box) * bl->cap);
        bl->s = realloc(bl->s, sizeof(orc_box) * bl->cap);
        bl->far = realloc(bl->far, sizeof(int) * bl->cap);
    }
    bl->t[bl->nblk] = *t;
    bl->s[bl->nblk] = *s;
    bl->far[bl->nblk] = far;
    bl->nblk++;
}

/* Statistics gathered while walking, for the structural pins. */
typedef struct {
    int64_t far_per_level[32];
    int64_t near;
    double storage;     /* doubles, paper layout: per far block p_eff^{2d} + factors;
                           per near block |tau| |sigma| */
} orc_walkstats;

static void children_walk(const orc_problem *P, int L, int p, double eta, const orc_box *t,
                          const orc_box *s, blist *bl, orc_walkstats *st)
{
    int d = P->d;
    if (admissible(d, t, s, eta)) {
        if (bl) blist_push(bl, t, s, 1);
        if (st) {
            st->far_per_level[t->level]++;
            double core = 1.0, fac = 0.0;
            for (int l = 0; l < d; ++l) {
                int pt = t->cnt[l] < p ? t->cnt[l] : p;
                int ps = s->cnt[l] < p ? s->cnt[l] : p;
                core *= (double)pt * ps;
                fac += (double)t->cnt[l] * pt + (double)s->cnt[l] * ps;
            }
            st->storage += core + fac;
        }
        return;
    }
    if (t->level == L || s->level == L) {   /* a leaf has no children */
        if (bl) blist_push(bl, t, s, 0);
        if (st) {
            st->near++;
            double a = 1.0, b = 1.0;
            for (int l = 0; l < d; ++l) { a *= t->cnt[l]; b *= s->cnt[l]; }
            st->storage += a * b;
        }
        return;
    }
    int nc = 1 << d;
    for (int ct = 0; ct < nc; ++ct) {
        int bt[3] = {0, 0, 0};
        for (int l = 0; l < d; ++l) bt[l] = 2 * t->b[l] + ((ct >> l) & 1);
        orc_box tc;
        make_box(P, t->level + 1, bt, &tc);
        for (int cs = 0; cs < nc; ++cs) {
            int bs[3] = {0, 0, 0};
            for (int l = 0; l < d; ++l) bs[l] = 2 * s->b[l] + ((cs >> l) & 1);
            orc_box sc;
            make_box(P, s->level + 1, bs, &sc);
            children_walk(P, L, p, eta, &tc, &sc, bl, st);
        }
    }
}

static int tree_depth(int n, int leaf)
{
    if (leaf < 1 || n % leaf) return -1;
    int r = n / leaf, L = 0;
    while (r > 1) {
        if (r & 1) return -1;
        r >>= 1;
        ++L;
    }
    return L;
}

/* Uniform grid x_i = (i + 1/2) h, cells [i h, (i+1) h] (Example 2.1), d dims. */
static void uniform_arrays(int d, int n, double *xb, double *eb)
{
    double h = 1.0 / n;
    for (int l = 0; l < d; ++l) {
        for (int i = 0; i < n; ++i) xb[l * n + i] = (i + 0.5) * h;
        for (int i = 0; i <= n; ++i) eb[l * (n + 1) + i] = i * h;
    }
}

/* Block-tree counts on a uniform grid, for the storage pins (Tables 5.1-5.4). */
int orc_htlr_count(int d, int n, int leaf, int p, double eta, int64_t *far_per_level,
                   int64_t *near, double *storage_doubles)
{
    int L = tree_depth(n, leaf);
    if (L < 0 || d < 1 || d > 3) return -1;
    double *xb = malloc(sizeof(double) * d * n), *eb = malloc(sizeof(double) * d * (n + 1));
    uniform_arrays(d, n, xb, eb);
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.d = d; P.n = n; P.uniform = 1;
    for (int l = 0; l < d; ++l) { P.x[l] = xb + l * n; P.edge[l] = eb + l * (n + 1); }
    setup_boxes(&P, L);
    orc_walkstats st;
    memset(&st, 0, sizeof st);
    int b0[3] = {0, 0, 0};
    orc_box root;
    make_box(&P, 0, b0, &root);
    children_walk(&P, L, p, eta, &root, &root, NULL, &st);
    for (int l = 0; l <= L; ++l) far_per_level[l] = st.far_per_level[l];
    *near = st.near;
    *storage_doubles = st.storage;
    free_boxes(&P);
    free(xb);
    free(eb);
    return L;
}

/* ------------------------------------------------------------------------------ */
/* Algorithm 1, Construct                                                          */
/* ------------------------------------------------------------------------------ */

/* Mode product on a tensor with dims[0..nd-1] (first index fastest): contracts mode
 * `mode` (size dims[mode]) with M (rows x dims[mode], column-major), producing a tensor
 * whose mode `mode` has size rows.  out = X x_mode M. */
static double *mode_product(const double *X, int nd, const int *dims, int mode,
                            const double *M, int rows, int *odims)
{
    long inner = 1, outer = 1;
    for (int k = 0; k < mode; ++k) inner *= dims[k];
    for (int k = mode + 1; k < nd; ++k) outer *= dims[k];
    int m = dims[mode];
    double *Y = calloc((size_t)inner * rows * outer, sizeof(double));
    for (long o = 0; o < outer; ++o)
        for (int r = 0; r < rows; ++r)
            for (long i = 0; i < inner; ++i) {
                double s = 0.0;
                for (int k = 0; k < m; ++k)
                    s += M[r + (long)k * rows] * X[i + inner * (k + (long)m * o)];
                Y[i + inner * (r + (long)rows * o)] = s;
            }
    for (int k = 0; k < nd; ++k) odims[k] = dims[k];
    odims[mode] = rows;
    return Y;
}

/* Interpolation factor (eq. (3.5)): F(i, mu) = L_mu(x_{first+i}) on the cell [lo, hi],
 * optionally times the 1-D cell width (tensor grids). */
static double *interp_factor(const orc_problem *P, int l, const orc_box *B, int p,
                             int with_width)
{
    double xi[64];
    orc_cheb_nodes(p, B->lo[l], B->hi[l], xi);
    int m = B->cnt[l];
    double *F = malloc(sizeof(double) * m * p);
    for (int i = 0; i < m; ++i) {
        int g = B->first[l] + i;
        double xv = P->x[l][g];
        double wv = with_width ? (P->edge[l][g + 1] - P->edge[l][g]) : 1.0;
        for (int mu = 0; mu < p; ++mu) F[i + (long)mu * m] = orc_lagrange(p, xi, mu, xv) * wv;
    }
    return F;
}

static void build_far(const orc_problem *P, int p, int orth, orc_block *K)
{
    int d = P->d;
    const orc_box *t = &K->tau, *s = &K->sig;
    int fold = !P->uniform;   /* tensor grids: widths folded into V */
    /* factors and core by Chebyshev interpolation, eq. (3.5) */
    double xt[3][64], xs[3][64];
    for (int l = 0; l < d; ++l) {
        orc_cheb_nodes(p, t->lo[l], t->hi[l], xt[l]);
        orc_cheb_nodes(p, s->lo[l], s->hi[l], xs[l]);
    }
    long pd = 1;
    for (int l = 0; l < d; ++l) pd *= p;
    double *G = malloc(sizeof(double) * pd * pd);
    double w = 1.0;
    if (P->uniform) w = pow(1.0 / P->n, d);   /* h^d, Algorithm 1 core update */
    for (long js = 0; js < pd; ++js)
        for (long it = 0; it < pd; ++it) {
            double xa[3], ya[3];
            long a = it, b = js;
            for (int l = 0; l < d; ++l) {
                xa[l] = xt[l][a % p]; a /= p;
                ya[l] = xs[l][b % p]; b /= p;
            }
            G[it + pd * js] = w * orc_kernel(P, xa, ya);
        }
    int dims[6];
    for (int k = 0; k < 2 * d; ++k) dims[k] = p;
    for (int l = 0; l < d; ++l) {
        double *Ul = interp_factor(P, l, t, p, 0);
        double *Vl = interp_factor(P, l, s, p, fold);
        if (orth) {
            /* U_l = W_l R_l, V_l = Q_l T_l; G <- G x_l R_l x_{d+l} T_l */
            int mt = t->cnt[l], ms = s->cnt[l];
            int kt = mt < p ? mt : p, ks = ms < p ? ms : p;
            double *W = malloc(sizeof(double) * mt * kt), *R = malloc(sizeof(double) * kt * p);
            double *Q = malloc(sizeof(double) * ms * ks), *T = malloc(sizeof(double) * ks * p);
            orc_qr(mt, p, Ul, W, R);
            orc_qr(ms, p, Vl, Q, T);
            int od[6];
            double *G1 = mode_product(G, 2 * d, dims, l, R, kt, od);
            free(G);
            memcpy(dims, od, sizeof od);
            double *G2 = mode_product(G1, 2 * d, dims, d + l, T, ks, od);
            free(G1);
            memcpy(dims, od, sizeof od);
            G = G2;
            free(Ul); free(Vl); free(R); free(T);
            K->U[l] = W; K->V[l] = Q; K->pt[l] = kt; K->ps[l] = ks;
        } else {
            K->U[l] = Ul; K->V[l] = Vl; K->pt[l] = p; K->ps[l] = p;
        }
    }
    K->G = G;
}

static void build_near(const orc_problem *P, orc_block *K)
{
    int d = P->d;
    const orc_box *t = &K->tau, *s = &K->sig;
    long nt = 1, ns = 1;
    for (int l = 0; l < d; ++l) { nt *= t->cnt[l]; ns *= s->cnt[l]; }
    K->D = malloc(sizeof(double) * nt * ns);
    /* eq. (4.1): A_ij = a(x_i) delta_ij + K_ij |Omega_j| */
    for (long js = 0; js < ns; ++js) {
        int mj[3];
        long b = js, gj = 0, str = 1;
        double y[3];
        for (int l = 0; l < d; ++l) {
            mj[l] = s->first[l] + (int)(b % s->cnt[l]);
            b /= s->cnt[l];
            y[l] = P->x[l][mj[l]];
            gj += mj[l] * str;
            str *= P->n;
        }
        double wj = cell_measure(P, mj);
        for (long it = 0; it < nt; ++it) {
            int mi[3];
            long a = it, gi = 0;
            str = 1;
            double x[3];
            for (int l = 0; l < d; ++l) {
                mi[l] = t->first[l] + (int)(a % t->cnt[l]);
                a /= t->cnt[l];
                x[l] = P->x[l][mi[l]];
                gi += mi[l] * str;
                str *= P->n;
            }
            double v;
            if (gi == gj) {
                double lo[3], hi[3];
                for (int l = 0; l < d; ++l) {
                    lo[l] = P->edge[l][mi[l]];
                    hi[l] = P->edge[l][mi[l] + 1];
                }
                v = orc_diag_integral(P, x, lo, hi) + (P->a ? P->a[gi] : 0.0);
            } else {
                v = orc_kernel(P, x, y) * wj;
            }
            K->D[it + nt * js] = v;
        }
    }
}

static void copy_problem(orc_htlr *H, int d, int n, int ktype, double kscale,
                         double kparam, const double *x, const double *edge,
                         const double *a, int uniform, int q)
{
    long N = 1;
    for (int l = 0; l < d; ++l) N *= n;
    H->xbuf = malloc(sizeof(double) * d * n);
    H->ebuf = malloc(sizeof(double) * d * (n + 1));
    if (x) {
        memcpy(H->xbuf, x, sizeof(double) * d * n);
        memcpy(H->ebuf, edge, sizeof(double) * d * (n + 1));
    } else {
        uniform_arrays(d, n, H->xbuf, H->ebuf);
    }
    H->abuf = NULL;
    if (a) {
        H->abuf = malloc(sizeof(double) * N);
        memcpy(H->abuf, a, sizeof(double) * N);
    }
    orc_problem *P = &H->P;
    memset(P, 0, sizeof *P);
    P->d = d; P->n = n; P->ktype = ktype; P->kscale = kscale; P->kparam = kparam;
    for (int l = 0; l < d; ++l) { P->x[l] = H->xbuf + l * n; P->edge[l] = H->ebuf + l * (n + 1); }
    P->a = H->abuf;
    P->uniform = uniform;
    P->q = q;
}

/* Construct (Algorithm 1).  x, edge: d*n and d*(n+1) arrays (dimension-major), or NULL
 * for the uniform grid of Example 2.1.  a: N values or NULL.  eta <= 0: weak.
 * Returns NULL on invalid arguments. */
orc_htlr *orc_htlr_construct(int d, int n, int ktype, double kscale, double kparam,
                             const double *x, const double *edge, const double *a,
                             int leaf, int p, double eta, int orth, int q)
{
    int L = tree_depth(n, leaf);
    if (L < 0 || d < 2 || d > 3 || p < 1 || p > 64 || q < 1) return NULL;
    orc_htlr *H = calloc(1, sizeof *H);
    copy_problem(H, d, n, ktype, kscale, kparam, x, edge, a, x == NULL, q);
    H->L = L; H->p = p; H->eta = eta; H->orth = orth;
    setup_boxes(&H->P, L);
    if (!boxes_nonempty(&H->P)) {
        orc_htlr_free(H);
        return NULL;
    }
    blist bl;
    memset(&bl, 0, sizeof bl);
    int b0[3] = {0, 0, 0};
    orc_box root;
    make_box(&H->P, 0, b0, &root);
    children_walk(&H->P, L, p, eta, &root, &root, &bl, NULL);
    H->nblk = bl.nblk;
    H->blk = calloc(bl.nblk, sizeof(orc_block));
    for (long k = 0; k < bl.nblk; ++k) {
        H->blk[k].tau = bl.t[k];
        H->blk[k].sig = bl.s[k];
        H->blk[k].far = bl.far[k];
    }
    free(bl.t); free(bl.s); free(bl.far);
    /* every block is built independently of the others */
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < H->nblk; ++k) {
        if (H->blk[k].far) build_far(&H->P, p, orth, &H->blk[k]);
        else build_near(&H->P, &H->blk[k]);
    }
    return H;
}

void orc_htlr_free(orc_htlr *H)
{
    if (!H) return;
    for (long k = 0; k < H->nblk; ++k) {
        orc_block *K = &H->blk[k];
        for (int l = 0; l < 3; ++l) { free(K->U[l]); free(K->V[l]); }
        free(K->G);
        free(K->D);
    }
    free(H->blk);
    free_boxes(&H->P);
    free(H->xbuf); free(H->ebuf); free(H->abuf);
    free(H);
}

/* Counts of the constructed structure: far per level (L+1 entries), near, and the
 * doubles actually stored by the oracle. */
int orc_htlr_stats(const orc_htlr *H, int64_t *far_per_level, int64_t *near,
                   double *stored_doubles)
{
    int d = H->P.d;
    for (int l = 0; l <= H->L; ++l) far_per_level[l] = 0;
    *near = 0;
    double st = 0;
    for (long k = 0; k < H->nblk; ++k) {
        const orc_block *K = &H->blk[k];
        if (K->far) {
            far_per_level[K->tau.level]++;
            double core = 1.0, fac = 0.0;
            for (int l = 0; l < d; ++l) {
                core *= (double)K->pt[l] * K->ps[l];
                fac += (double)K->tau.cnt[l] * K->pt[l] + (double)K->sig.cnt[l] * K->ps[l];
            }
            st += core + fac;
        } else {
            (*near)++;
            double a = 1, b = 1;
            for (int l = 0; l < d; ++l) { a *= K->tau.cnt[l]; b *= K->sig.cnt[l]; }
            st += a * b;
        }
    }
    *stored_doubles = st;
    return H->L;
}

/* ------------------------------------------------------------------------------ */
/* Algorithm 2, HMultVec                                                            */
/* ------------------------------------------------------------------------------ */

/* Gather u_sigma (reshaped to a d-tensor, eq. (4.3)) for one right-hand side. */
static void gather_box(const orc_problem *P, const orc_box *B, const double *u, double *out)
{
    long m = 1;
    for (int l = 0; l < P->d; ++l) m *= B->cnt[l];
    for (long j = 0; j < m; ++j) {
        long b = j, g = 0, str = 1;
        for (int l = 0; l < P->d; ++l) {
            g += (B->first[l] + b % B->cnt[l]) * str;
            b /= B->cnt[l];
            str *= P->n;
        }
        out[j] = u[g];
    }
}

static void scatter_add_box(const orc_problem *P, const orc_box *B, const double *v,
                            double *f)
{
    long m = 1;
    for (int l = 0; l < P->d; ++l) m *= B->cnt[l];
    for (long j = 0; j < m; ++j) {
        long b = j, g = 0, str = 1;
        for (int l = 0; l < P->d; ++l) {
            g += (B->first[l] + b % B->cnt[l]) * str;
            b /= B->cnt[l];
            str *= P->n;
        }
        f[g] += v[j];
    }
}

/* v = A_{tau,sigma} u_sigma for one block (the two leaf cases of Algorithm 2); v has
 * |tau| entries in the box's local order (first index fastest). */
static void block_product(const orc_problem *P, const orc_block *K, const double *u, double *v)
{
    int d = P->d;
    const orc_box *t = &K->tau, *s = &K->sig;
    long nt = 1, ns = 1;
    for (int l = 0; l < d; ++l) { nt *= t->cnt[l]; ns *= s->cnt[l]; }
    double *us = malloc(sizeof(double) * ns);
    gather_box(P, s, u, us);
    if (K->far) {
        /* W = U_sigma x_1 V_1^T ... x_d V_d^T */
        int dims[3];
        for (int l = 0; l < d; ++l) dims[l] = s->cnt[l];
        double *W = us;
        for (int l = 0; l < d; ++l) {
            int m = s->cnt[l], r = K->ps[l];
            double *VT = malloc(sizeof(double) * r * m);
            for (int i = 0; i < m; ++i)
                for (int c = 0; c < r; ++c) VT[c + (long)i * r] = K->V[l][i + (long)c * m];
            int od[3];
            double *W2 = mode_product(W, d, dims, l, VT, r, od);
            free(VT);
            free(W);
            W = W2;
            memcpy(dims, od, sizeof od);
        }
        /* H = G x_{[d+1..2d],[1..d]} W */
        long pt = 1, ps = 1;
        for (int l = 0; l < d; ++l) { pt *= K->pt[l]; ps *= K->ps[l]; }
        double *Hv = calloc(pt, sizeof(double));
        for (long it = 0; it < pt; ++it) {
            double acc = 0.0;
            for (long js = 0; js < ps; ++js) acc += K->G[it + pt * js] * W[js];
            Hv[it] = acc;
        }
        free(W);
        /* F = H x_1 U_1 ... x_d U_d */
        for (int l = 0; l < d; ++l) dims[l] = K->pt[l];
        double *F = Hv;
        for (int l = 0; l < d; ++l) {
            int od[3];
            double *F2 = mode_product(F, d, dims, l, K->U[l], t->cnt[l], od);
            free(F);
            F = F2;
            memcpy(dims, od, sizeof od);
        }
        memcpy(v, F, sizeof(double) * nt);
        free(F);
    } else {
        for (long it = 0; it < nt; ++it) v[it] = 0.0;
        for (long js = 0; js < ns; ++js)
            for (long it = 0; it < nt; ++it) v[it] += K->D[it + nt * js] * us[js];
        free(us);
    }
}

/* f_tau += A_{tau,sigma} u_sigma for one block. */
static void apply_block(const orc_problem *P, const orc_block *K, const double *u, double *f)
{
    long nt = 1;
    for (int l = 0; l < P->d; ++l) nt *= K->tau.cnt[l];
    double *v = malloc(sizeof(double) * nt);
    block_product(P, K, u, v);
    scatter_add_box(P, &K->tau, v, f);
    free(v);
}

/* HMultVec (Algorithm 2) from the root: f = A u (f starts at zero), column by column.
 * The blocks are visited in the order of the block-tree recursion.  Serially that is
 * f_tau += A_{tau,sigma} u_sigma block after block.  Here the per-block products run on
 * all host cores (OpenMP), each into its own buffer; then every leaf box of the tree
 * gathers, in recursion order, the contributions of the blocks whose target box
 * contains it.  Each element of f thus receives the same additions in the same order as
 * in the serial loop, and the result is bitwise independent of the thread count. */
int orc_htlr_matvec(const orc_htlr *H, const double *u, int nrhs, double *f)
{
    const orc_problem *P = &H->P;
    const int d = P->d, L = H->L;
    long N = 1;
    for (int l = 0; l < d; ++l) N *= P->n;
    const long nblk = H->nblk;
    long *off = malloc(sizeof(long) * (nblk + 1));
    off[0] = 0;
    for (long k = 0; k < nblk; ++k) {
        long nt = 1;
        for (int l = 0; l < d; ++l) nt *= H->blk[k].tau.cnt[l];
        off[k + 1] = off[k] + nt;
    }
    double *buf = malloc(sizeof(double) * (off[nblk] > 0 ? off[nblk] : 1));
    /* per leaf box: the blocks whose target box contains it, in recursion order */
    const int nl1 = 1 << L;
    long nleaf = 1;
    for (int l = 0; l < d; ++l) nleaf *= nl1;
    long *lcnt = calloc(nleaf + 1, sizeof(long));
    for (long k = 0; k < nblk; ++k) {
        const orc_box *t = &H->blk[k].tau;
        const int sh = L - t->level, w = 1 << sh;
        long span = 1;
        for (int l = 0; l < d; ++l) span *= w;
        for (long q = 0; q < span; ++q) {
            long rem = q, leaf = 0, str = 1;
            for (int l = 0; l < d; ++l) {
                leaf += (long)((t->b[l] << sh) + rem % w) * str;
                rem /= w;
                str *= nl1;
            }
            lcnt[leaf + 1]++;
        }
    }
    for (long b = 0; b < nleaf; ++b) lcnt[b + 1] += lcnt[b];
    long *lblk = malloc(sizeof(long) * (lcnt[nleaf] > 0 ? lcnt[nleaf] : 1));
    long *fill = malloc(sizeof(long) * (nleaf > 0 ? nleaf : 1));
    for (long b = 0; b < nleaf; ++b) fill[b] = lcnt[b];
    for (long k = 0; k < nblk; ++k) {          /* increasing k: lists in recursion order */
        const orc_box *t = &H->blk[k].tau;
        const int sh = L - t->level, w = 1 << sh;
        long span = 1;
        for (int l = 0; l < d; ++l) span *= w;
        for (long q = 0; q < span; ++q) {
            long rem = q, leaf = 0, str = 1;
            for (int l = 0; l < d; ++l) {
                leaf += (long)((t->b[l] << sh) + rem % w) * str;
                rem /= w;
                str *= nl1;
            }
            lblk[fill[leaf]++] = k;
        }
    }
    free(fill);
    for (int c = 0; c < nrhs; ++c) {
        const double *uc = u + (long)c * N;
        double *fc = f + (long)c * N;
        memset(fc, 0, sizeof(double) * N);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (long k = 0; k < nblk; ++k) block_product(P, &H->blk[k], uc, buf + off[k]);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (long b = 0; b < nleaf; ++b) {
            int bl[3] = {0, 0, 0};
            long rem = b;
            for (int l = 0; l < d; ++l) { bl[l] = (int)(rem % nl1); rem /= nl1; }
            orc_box lf;
            make_box(P, L, bl, &lf);
            for (long e = lcnt[b]; e < lcnt[b + 1]; ++e) {
                const long k = lblk[e];
                const orc_box *t = &H->blk[k].tau;
                const double *v = buf + off[k];
                /* every point of the leaf: its index in the target box and in f */
                for (int i3 = 0; i3 < lf.cnt[2]; ++i3)
                    for (int i2 = 0; i2 < lf.cnt[1]; ++i2)
                        for (int i1 = 0; i1 < lf.cnt[0]; ++i1) {
                            const int gi[3] = {lf.first[0] + i1, lf.first[1] + i2,
                                               lf.first[2] + i3};
                            long g = 0, gs = 1, j = 0, js = 1;
                            for (int l = 0; l < d; ++l) {
                                g += gi[l] * gs;
                                gs *= P->n;
                                j += (gi[l] - t->first[l]) * js;
                                js *= t->cnt[l];
                            }
                            fc[g] += v[j];
                        }
            }
        }
    }
    free(lblk);
    free(lcnt);
    free(buf);
    free(off);
    return 0;
}

/* Thread count of the oracle's OpenMP loops (n <= 0: the OpenMP default).  Returns the
 * count now in effect. */
int orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------------ */
/* Row-sampled HTLR (for grids too large to store): rows[] of f = A u.  Every block  */
/* whose target box holds a sampled row is built by Algorithm 1 and applied by       */
/* Algorithm 2; only the sampled rows of the result are kept.                         */
/* ------------------------------------------------------------------------------ */
static int box_has_row(const orc_problem *P, const orc_box *B, long row)
{
    long r = row;
    for (int l = 0; l < P->d; ++l) {
        int i = (int)(r % P->n);
        r /= P->n;
        if (i < B->first[l] || i >= B->first[l] + B->cnt[l]) return 0;
    }
    return 1;
}

static void rows_walk(const orc_problem *P, int L, double eta, const orc_box *t,
                      const orc_box *s, const int64_t *rows, int64_t nrows, blist *bl)
{
    int hit = 0;
    for (int64_t r = 0; r < nrows && !hit; ++r) hit = box_has_row(P, t, (long)rows[r]);
    if (!hit) return;
    if (admissible(P->d, t, s, eta)) { blist_push(bl, t, s, 1); return; }
    if (t->level == L || s->level == L) { blist_push(bl, t, s, 0); return; }
    int nc = 1 << P->d;
    for (int ct = 0; ct < nc; ++ct) {
        int bt[3] = {0, 0, 0};
        for (int l = 0; l < P->d; ++l) bt[l] = 2 * t->b[l] + ((ct >> l) & 1);
        orc_box tc;
        make_box(P, t->level + 1, bt, &tc);
        for (int cs = 0; cs < nc; ++cs) {
            int bs[3] = {0, 0, 0};
            for (int l = 0; l < P->d; ++l) bs[l] = 2 * s->b[l] + ((cs >> l) & 1);
            orc_box sc;
            make_box(P, s->level + 1, bs, &sc);
            rows_walk(P, L, eta, &tc, &sc, rows, nrows, bl);
        }
    }
}

int orc_htlr_rows(int d, int n, int ktype, double kscale, double kparam, const double *x,
                  const double *edge, const double *a, int leaf, int p, double eta, int orth,
                  int q, const double *u, int nrhs, const int64_t *rows, int64_t nrows,
                  double *frows)
{
    int L = tree_depth(n, leaf);
    if (L < 0 || d < 2 || d > 3 || p < 1 || p > 64) return -1;
    orc_htlr H;
    memset(&H, 0, sizeof H);
    copy_problem(&H, d, n, ktype, kscale, kparam, x, edge, a, x == NULL, q);
    setup_boxes(&H.P, L);
    if (!boxes_nonempty(&H.P)) {
        free_boxes(&H.P);
        free(H.xbuf); free(H.ebuf); free(H.abuf);
        return -1;
    }
    const orc_problem *P = &H.P;
    long N = 1;
    for (int l = 0; l < d; ++l) N *= n;
    blist bl;
    memset(&bl, 0, sizeof bl);
    int b0[3] = {0, 0, 0};
    orc_box root;
    make_box(P, 0, b0, &root);
    rows_walk(P, L, eta, &root, &root, rows, nrows, &bl);
    for (long k = 0; k < (long)nrows * nrhs; ++k) frows[k] = 0.0;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    /* per-thread partial results, summed at the end in thread order */
    double *part = calloc((size_t)nth * nrows * nrhs, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *fl = calloc(N, sizeof(double));
        double *mine = part + (size_t)tid * nrows * nrhs;
#pragma omp for schedule(dynamic, 1)
        for (long k = 0; k < bl.nblk; ++k) {
            orc_block K;
            memset(&K, 0, sizeof K);
            K.tau = bl.t[k]; K.sig = bl.s[k]; K.far = bl.far[k];
            if (K.far) build_far(P, p, orth, &K);
            else build_near(P, &K);
            long nt = 1;
            for (int l = 0; l < d; ++l) nt *= K.tau.cnt[l];
            for (int c = 0; c < nrhs; ++c) {
                /* f_tau = A_{tau,sigma} u_sigma into a zeroed scratch vector */
                apply_block(P, &K, u + (long)c * N, fl);
                for (int64_t r = 0; r < nrows; ++r)
                    if (box_has_row(P, &K.tau, (long)rows[r])) {
                        mine[r + (long)c * nrows] += fl[rows[r]];
                    }
                /* clear the target box again */
                long m = nt;
                for (long j = 0; j < m; ++j) {
                    long b = j, g = 0, str = 1;
                    for (int l = 0; l < d; ++l) {
                        g += (K.tau.first[l] + b % K.tau.cnt[l]) * str;
                        b /= K.tau.cnt[l];
                        str *= n;
                    }
                    fl[g] = 0.0;
                }
            }
            for (int l = 0; l < 3; ++l) { free(K.U[l]); free(K.V[l]); }
            free(K.G);
            free(K.D);
        }
        free(fl);
    }
    for (int t = 0; t < nth; ++t)
        for (long k = 0; k < (long)nrows * nrhs; ++k) frows[k] += part[(size_t)t * nrows * nrhs + k];
    free(part);
    free(bl.t); free(bl.s); free(bl.far);
    free_boxes(&H.P);
    free(H.xbuf); free(H.ebuf); free(H.abuf);
    return 0;
}

/* Number of OpenMP threads the oracle uses (reported beside its timings). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Build one far block (Algorithm 1, admissible leaf) between the level-`level` boxes
 * bt and bs and return its factors and core, for the unit pins.  U: d blocks of
 * cnt x pt (concatenated), V likewise, G: prod pt x prod ps.  Returns 0 if the pair is
 * admissible, 1 if not (nothing written), -1 on bad arguments. */
int orc_far_block(int d, int n, int ktype, double kscale, double kparam, const double *x,
                  const double *edge, int level, const int *bt, const int *bs, int p,
                  double eta, int orth, int *pt, int *ps, double *U, double *V, double *G)
{
    if (d < 1 || d > 3 || p < 1 || p > 64) return -1;
    orc_htlr H;
    memset(&H, 0, sizeof H);
    copy_problem(&H, d, n, ktype, kscale, kparam, x, edge, NULL, x == NULL, 8);
    setup_boxes(&H.P, level);
    orc_block K;
    memset(&K, 0, sizeof K);
    make_box(&H.P, level, bt, &K.tau);
    make_box(&H.P, level, bs, &K.sig);
    int rc = 1;
    if (admissible(d, &K.tau, &K.sig, eta)) {
        build_far(&H.P, p, orth, &K);
        long offu = 0, offv = 0, nt = 1, ns = 1;
        for (int l = 0; l < d; ++l) {
            pt[l] = K.pt[l];
            ps[l] = K.ps[l];
            memcpy(U + offu, K.U[l], sizeof(double) * K.tau.cnt[l] * K.pt[l]);
            memcpy(V + offv, K.V[l], sizeof(double) * K.sig.cnt[l] * K.ps[l]);
            offu += (long)K.tau.cnt[l] * K.pt[l];
            offv += (long)K.sig.cnt[l] * K.ps[l];
            nt *= K.pt[l];
            ns *= K.ps[l];
        }
        memcpy(G, K.G, sizeof(double) * nt * ns);
        rc = 0;
    }
    for (int l = 0; l < 3; ++l) { free(K.U[l]); free(K.V[l]); }
    free(K.G);
    free_boxes(&H.P);
    free(H.xbuf); free(H.ebuf); free(H.abuf);
    return rc;
}

/* Rows of the dense Nystrom product with plain arguments (x, edge NULL: uniform grid). */
int orc_dense_rows_api(int d, int n, int ktype, double kscale, double kparam,
                       const double *x, const double *edge, const double *a, int q,
                       const double *u, int nrhs, const int64_t *rows, int64_t nrows,
                       double *frows)
{
    if (d < 1 || d > 3 || n < 1 || q < 1) return -1;
    orc_htlr H;
    memset(&H, 0, sizeof H);
    copy_problem(&H, d, n, ktype, kscale, kparam, x, edge, a, x == NULL, q);
    long N = 1;
    for (int l = 0; l < d; ++l) N *= n;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= N) {
            free(H.xbuf); free(H.ebuf); free(H.abuf);
            return -1;
        }
    int rc = orc_dense_rows(&H.P, u, nrhs, rows, nrows, frows);
    free(H.xbuf); free(H.ebuf); free(H.abuf);
    return rc;
}

/* Algorithm 2 restricted to the blocks k0..k1-1 (recursion order), accumulated into f
 * for one right-hand side (f is not cleared).  Returns the multiply-adds of the core and
 * dense products of those blocks, so that a timed slice can be scaled to the whole
 * product; a bounded sample of the full HMultVec. */
double orc_htlr_matvec_range(const orc_htlr *H, const double *u, double *f, long k0, long k1)
{
    double work = 0.0;
    int d = H->P.d;
    if (k0 < 0) k0 = 0;
    if (k1 > H->nblk) k1 = H->nblk;
    for (long k = k0; k < k1; ++k) {
        const orc_block *K = &H->blk[k];
        apply_block(&H->P, K, u, f);
        double a = 1.0, b = 1.0;
        for (int l = 0; l < d; ++l) {
            if (K->far) { a *= K->pt[l]; b *= K->ps[l]; }
            else { a *= K->tau.cnt[l]; b *= K->sig.cnt[l]; }
        }
        work += a * b;
    }
    return work;
}

long orc_htlr_nblocks(const orc_htlr *H) { return H->nblk; }
