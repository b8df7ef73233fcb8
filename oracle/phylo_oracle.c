/*
 * phylo_oracle.c -- plain, slow FP64 CPU oracle for the phylogenetic log-likelihood and its
 * branch-length gradient (Ji et al., "Gradients do grow on trees", arXiv 1905.12146).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline load this file.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, for one rooted tree with N tips (nodes 0..N-1) and internal nodes N..n-1
 * (root = the node whose parent is -1), m states, C discrete rate categories and P site patterns:
 *   P_{i,l}  = e^{Q_i b_i r_l}                                   (Section 2.1; Section 2.5)
 *   p_k      = (P_{i,l} p_i) o (P_{j,l} p_j)   post-order        (Section 2.3, post-order update)
 *   L_p      = sum_l w_l pi' p_root,l                            (Section 2.3 root inner product;
 *                                                                 Section 2.5 mixture)
 *   q_root   = pi;  q_i = P_{i,l}' [q_k o (P_{j,l} p_j)]   pre-order (Section 2.4)
 * The paper's tree is binary (n = 2N-1, Section 2.1).  A node with more than two children
 * (a multifurcation) takes the same updates with the sibling set widened: p_k is the product of
 * P_c p_c over all its children c, and q_i multiplies q_k by P_s p_s for every sibling s of i.
 *   dlogL/db_i = sum_p wt_p sum_l r_l w_l p_i,l' Q_i' q_i,l / L_p      (Section 2.5 gradient with
 *                                                                 rate categories)
 *   d2logL/db_i^2 = sum_p wt_p [ sum_l r_l^2 w_l p' (Q_i^2)' q / L_p - (per-site gradient)^2 ]
 *                                                                (Section 2.6 Hessian diagonal,
 *                                                                 applied site by site)
 *   logL     = sum_p wt_p log L_p  (sites i.i.d., Section 2.1)
 *
 * Underflow (the paper is silent): after every node update the vector of a pattern (all
 * categories and states) is multiplied by an exact power of two so that its largest entry lies
 * in [0.5, 1); the integer log2 factors are carried alongside.  Multiplying by 2^k is exact, so
 * the result equals the unscaled definition up to rounding.
 *
 * Matrix exponential (the paper is silent on the method): diagonal Pade approximant of degree 8
 * with scaling and squaring (Moler & Van Loan 1978; Higham 2005), written here from the
 * definition of the [q/q] Pade coefficients, with ||A||_1 scaled below 1/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_NOMEM 2

/* ----------------------------------------------------------------------------------------- */
/* dense helpers (row-major m x m)                                                           */
/* ----------------------------------------------------------------------------------------- */

static void mat_mul(int m, const double *A, const double *B, double *C)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int k = 0; k < m; ++k) s += A[i * m + k] * B[k * m + j];
            C[i * m + j] = s;
        }
}

/* Solve D X = N for X (m x m right-hand sides), Gaussian elimination with partial pivoting. */
static int solve_square(int m, double *D, double *N)
{
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(D[r * m + c]) > fabs(D[piv * m + c])) piv = r;
        if (D[piv * m + c] == 0.0) return ORC_INVALID;
        if (piv != c) {
            for (int k = 0; k < m; ++k) {
                double t = D[c * m + k]; D[c * m + k] = D[piv * m + k]; D[piv * m + k] = t;
                t = N[c * m + k]; N[c * m + k] = N[piv * m + k]; N[piv * m + k] = t;
            }
        }
        for (int r = c + 1; r < m; ++r) {
            double f = D[r * m + c] / D[c * m + c];
            if (f == 0.0) continue;
            for (int k = c; k < m; ++k) D[r * m + k] -= f * D[c * m + k];
            for (int k = 0; k < m; ++k) N[r * m + k] -= f * N[c * m + k];
        }
    }
    for (int c = m - 1; c >= 0; --c) {
        for (int k = 0; k < m; ++k) {
            double s = N[c * m + k];
            for (int j = c + 1; j < m; ++j) s -= D[c * m + j] * N[j * m + k];
            N[c * m + k] = s / D[c * m + c];
        }
    }
    return ORC_OK;
}

/* e^A for a general real m x m matrix A (no reversibility or symmetry assumed). */
int orc_expm(int m, const double *A, double *out)
{
    enum { Q_DEG = 8 };
    if (m <= 0) return ORC_INVALID;
    size_t mm = (size_t)m * m;
    double *X = malloc(mm * sizeof(double)), *Pk = malloc(mm * sizeof(double));
    double *T = malloc(mm * sizeof(double)), *Nm = malloc(mm * sizeof(double));
    double *Dm = malloc(mm * sizeof(double));
    if (!X || !Pk || !T || !Nm || !Dm) {
        free(X); free(Pk); free(T); free(Nm); free(Dm);
        return ORC_NOMEM;
    }
    /* 1-norm and scaling: ||A / 2^s||_1 <= 1/2 */
    double norm = 0.0;
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += fabs(A[i * m + j]);
        if (s > norm) norm = s;
    }
    int s = 0;
    while (norm > 0.5) { norm *= 0.5; ++s; }
    double scale = ldexp(1.0, -s);
    for (size_t t = 0; t < mm; ++t) X[t] = A[t] * scale;

    /* Pade coefficients c_k = (2q-k)! q! / ((2q)! k! (q-k)!) */
    double c[Q_DEG + 1];
    for (int k = 0; k <= Q_DEG; ++k) {
        double v = 1.0;
        for (int t = 2 * Q_DEG - k + 1; t <= 2 * Q_DEG; ++t) v /= (double)t;   /* (2q-k)!/(2q)! */
        for (int t = Q_DEG - k + 1; t <= Q_DEG; ++t) v *= (double)t;           /* q!/(q-k)!     */
        for (int t = 2; t <= k; ++t) v /= (double)t;                           /* 1/k!          */
        c[k] = v;
    }
    /* N = sum c_k X^k,  D = sum c_k (-X)^k */
    for (size_t t = 0; t < mm; ++t) { Pk[t] = 0.0; Nm[t] = 0.0; Dm[t] = 0.0; }
    for (int i = 0; i < m; ++i) Pk[i * m + i] = 1.0;
    for (int k = 0; k <= Q_DEG; ++k) {
        double sign = (k % 2 == 0) ? 1.0 : -1.0;
        for (size_t t = 0; t < mm; ++t) {
            Nm[t] += c[k] * Pk[t];
            Dm[t] += sign * c[k] * Pk[t];
        }
        if (k < Q_DEG) {
            mat_mul(m, Pk, X, T);
            memcpy(Pk, T, mm * sizeof(double));
        }
    }
    int rc = solve_square(m, Dm, Nm);   /* Nm <- D^{-1} N */
    if (rc == ORC_OK) {
        for (int t = 0; t < s; ++t) {
            mat_mul(m, Nm, Nm, T);
            memcpy(Nm, T, mm * sizeof(double));
        }
        memcpy(out, Nm, mm * sizeof(double));
    }
    free(X); free(Pk); free(T); free(Nm); free(Dm);
    return rc;
}

/* ----------------------------------------------------------------------------------------- */
/* tree                                                                                      */
/* ----------------------------------------------------------------------------------------- */

typedef struct {
    int n_nodes, n_tips, root;
    int *kid_off;       /* children of node k: kids[kid_off[k] .. kid_off[k+1]-1] (none for tips) */
    int *kids;          /* in increasing node order */
    int *order;         /* pre-order (parents before children); reversed = post-order */
} tree_t;

static void tree_free(tree_t *t)
{
    free(t->kid_off); free(t->kids); free(t->order);
}

/* Nodes 0..n_tips-1 are the tips, n_tips..n_nodes-1 internal; every internal node has at least two
 * children, tips none; one root; every node reachable from it. */
static int tree_build(int n_tips, int n_nodes, const int32_t *parent, tree_t *t)
{
    int n = n_nodes;
    memset(t, 0, sizeof(*t));
    if (n_tips < 2 || n < n_tips + 1 || n > 2 * n_tips - 1) return ORC_INVALID;
    t->n_nodes = n; t->n_tips = n_tips; t->root = -1;
    t->kid_off = calloc((size_t)n + 1, sizeof(int)); t->kids = malloc((size_t)n * sizeof(int));
    t->order = malloc((size_t)n * sizeof(int));
    if (!t->kid_off || !t->kids || !t->order) { tree_free(t); return ORC_NOMEM; }
    for (int i = 0; i < n; ++i) {
        int p = parent[i];
        if (p < 0) {
            if (t->root >= 0) { tree_free(t); return ORC_INVALID; }
            t->root = i;
            continue;
        }
        if (p >= n || p < n_tips || p == i) { tree_free(t); return ORC_INVALID; }
        t->kid_off[p + 1]++;
    }
    if (t->root < n_tips) { tree_free(t); return ORC_INVALID; }
    for (int k = 0; k < n; ++k) {
        int deg = t->kid_off[k + 1];
        if (k >= n_tips && deg < 2) { tree_free(t); return ORC_INVALID; }
        t->kid_off[k + 1] += t->kid_off[k];
    }
    int *fill = malloc((size_t)n * sizeof(int));
    if (!fill) { tree_free(t); return ORC_NOMEM; }
    for (int k = 0; k < n; ++k) fill[k] = t->kid_off[k];
    for (int i = 0; i < n; ++i)
        if (parent[i] >= 0) t->kids[fill[parent[i]]++] = i;
    /* depth-first pre-order from the root */
    int top = 0, cnt = 0;
    fill[top++] = t->root;   /* fill doubles as the stack */
    while (top > 0) {
        int k = fill[--top];
        if (cnt >= n) { free(fill); tree_free(t); return ORC_INVALID; }
        t->order[cnt++] = k;
        for (int c = t->kid_off[k + 1] - 1; c >= t->kid_off[k]; --c) {
            if (top >= n) { free(fill); tree_free(t); return ORC_INVALID; }
            fill[top++] = t->kids[c];
        }
    }
    free(fill);
    if (cnt != n) { tree_free(t); return ORC_INVALID; }   /* unreachable nodes: a cycle */
    return ORC_OK;
}

/* ----------------------------------------------------------------------------------------- */
/* likelihood, gradient, Hessian diagonal                                                    */
/* ----------------------------------------------------------------------------------------- */

/* Multiply the m*C values of one pattern by 2^-e so that the largest lies in [0.5, 1).  Returns
 * e (0 when every value is 0). */
static int rescale(double *v, int len)
{
    double mx = 0.0;
    for (int t = 0; t < len; ++t) if (v[t] > mx) mx = v[t];
    if (mx == 0.0 || !isfinite(mx)) return 0;
    int e;
    frexp(mx, &e);
    for (int t = 0; t < len; ++t) v[t] = ldexp(v[t], -e);
    return e;
}

/*
 * Inputs (host, FP64 unless stated), n = n_nodes (2N-1 for a binary tree, fewer with
 * multifurcations; tips are nodes 0..N-1, every internal node has at least two children):
 *   parent[n] (int32), tips[N][P] (uint8), weights[P], Q[n_models][m][m],
 *   branch_model[n] (NULL = model 0), pi[m], rates[C], cat_w[C], b[n] (root entry ignored),
 *   tip_vecs[K][m] (K = n_tip_vecs >= 0; NULL when K = 0).
 * A tip's partial vector at a pattern (Section 2.1) follows its code y: the indicator of state y
 * for y < m; row y - m of tip_vecs for m <= y < m + K (partially observed data: finite entries
 * >= 0, at least one positive); the all-ones vector (missing data) for y >= m + K.
 * Outputs: logL (scalar), grad[n] (root entry 0), site_logL[P], hess[n] (each may be NULL).
 * Optional introspection (NULL to skip): post[n][P][C][m] and pre[n][P][C][m] scaled partials
 * with their integer log2 factors post_e[n][P], pre_e[n][P] (value = stored * 2^e).
 */
int orc_eval_tree(int n_tips, int n_nodes, int m, int n_patterns, int n_cat, int n_models,
                  const int32_t *parent, const uint8_t *tips, const double *weights,
                  const double *Q, const int32_t *branch_model, const double *pi,
                  const double *rates, const double *cat_w, const double *b,
                  int n_tip_vecs, const double *tip_vecs,
                  double *logL, double *grad, double *site_logL, double *hess,
                  double *post_out, double *pre_out, int32_t *post_e_out, int32_t *pre_e_out)
{
    if (n_tips < 2 || m < 2 || n_patterns < 0 || n_cat < 1 || n_models < 1) return ORC_INVALID;
    if (n_tip_vecs < 0 || (n_tip_vecs > 0 && !tip_vecs)) return ORC_INVALID;
    for (int v = 0; v < n_tip_vecs; ++v) {
        int positive = 0;
        for (int s = 0; s < m; ++s) {
            const double x = tip_vecs[(size_t)v * m + s];
            if (!(x >= 0.0) || !isfinite(x)) return ORC_INVALID;
            if (x > 0.0) positive = 1;
        }
        if (!positive) return ORC_INVALID;
    }
    tree_t t;
    int rc = tree_build(n_tips, n_nodes, parent, &t);
    if (rc != ORC_OK) return rc;
    const int n = t.n_nodes, P = n_patterns, C = n_cat;
    const size_t mm = (size_t)m * m, row = (size_t)C * m;   /* row = one pattern of one node */
    for (int i = 0; i < n; ++i) {
        if (i != t.root && !(b[i] >= 0.0)) { tree_free(&t); return ORC_INVALID; }
        if (branch_model && (branch_model[i] < 0 || branch_model[i] >= n_models)) {
            tree_free(&t); return ORC_INVALID;
        }
    }

    double *Pm = calloc((size_t)n * C * mm, sizeof(double));      /* P_{i,l}           */
    double *post = calloc((size_t)n * P * row, sizeof(double));   /* p_i (scaled)      */
    double *pre = calloc((size_t)n * P * row, sizeof(double));    /* q_i (scaled)      */
    int32_t *pe = calloc((size_t)n * P, sizeof(int32_t));         /* log2 factor of p  */
    int32_t *qe = calloc((size_t)n * P, sizeof(int32_t));         /* log2 factor of q  */
    double *Lhat = calloc((size_t)P > 0 ? P : 1, sizeof(double)); /* L_p / 2^{pe_root} */
    double *A = malloc(mm * sizeof(double)), *Q2 = malloc(mm * sizeof(double));
    double *u = malloc(m * sizeof(double));
    if (!Pm || !post || !pre || !pe || !qe || !Lhat || !A || !Q2 || !u) {
        rc = ORC_NOMEM; goto done;
    }

    /* transition matrices P_{i,l} = exp(Q_i b_i r_l)  (Sections 2.1, 2.5) */
    for (int i = 0; i < n; ++i) {
        if (i == t.root) continue;
        const double *Qi = Q + (size_t)(branch_model ? branch_model[i] : 0) * mm;
        for (int l = 0; l < C; ++l) {
            for (size_t x = 0; x < mm; ++x) A[x] = Qi[x] * b[i] * rates[l];
            rc = orc_expm(m, A, Pm + ((size_t)i * C + l) * mm);
            if (rc != ORC_OK) goto done;
        }
    }

    /* post-order: tips are their partial vectors (indicator, given, or all-ones), internal nodes
     * by the pruning update */
    for (int o = n - 1; o >= 0; --o) {
        int k = t.order[o];
        for (int p = 0; p < P; ++p) {
            double *pk = post + ((size_t)k * P + p) * row;
            if (k < n_tips) {
                int y = tips[(size_t)k * P + p];
                for (int l = 0; l < C; ++l)
                    for (int s = 0; s < m; ++s) {
                        double v;
                        if (y < m) v = (y == s) ? 1.0 : 0.0;
                        else if (y < m + n_tip_vecs) v = tip_vecs[(size_t)(y - m) * m + s];
                        else v = 1.0;
                        pk[l * m + s] = v;
                    }
                pe[(size_t)k * P + p] = 0;
                continue;
            }
            /* p_k = product over the children c of P_c p_c (two children in the paper's
             * binary tree) */
            int ek = 0;
            for (size_t x = 0; x < row; ++x) pk[x] = 1.0;
            for (int o2 = t.kid_off[k]; o2 < t.kid_off[k + 1]; ++o2) {
                int c = t.kids[o2];
                const double *pc = post + ((size_t)c * P + p) * row;
                for (int l = 0; l < C; ++l) {
                    const double *Pc = Pm + ((size_t)c * C + l) * mm;
                    for (int s2 = 0; s2 < m; ++s2) {
                        double a = 0.0;
                        for (int x = 0; x < m; ++x) a += Pc[s2 * m + x] * pc[l * m + x];
                        pk[l * m + s2] *= a;
                    }
                }
                ek += pe[(size_t)c * P + p];
            }
            pe[(size_t)k * P + p] = ek + rescale(pk, (int)row);
        }
    }

    /* root: L_p = sum_l w_l pi' p_root,l ; logL = sum_p wt_p log L_p */
    double total = 0.0;
    for (int p = 0; p < P; ++p) {
        const double *pr = post + ((size_t)t.root * P + p) * row;
        double L = 0.0;
        for (int l = 0; l < C; ++l)
            for (int s = 0; s < m; ++s) L += cat_w[l] * pi[s] * pr[l * m + s];
        Lhat[p] = L;
        double lp = log(L) + (double)pe[(size_t)t.root * P + p] * log(2.0);
        if (site_logL) site_logL[p] = lp;
        total += weights[p] * lp;
    }
    if (logL) *logL = total;

    /* pre-order: q_root = pi, q_i = P_i' [q_k o (P_j p_j)] */
    for (int p = 0; p < P; ++p) {
        double *qr = pre + ((size_t)t.root * P + p) * row;
        for (int l = 0; l < C; ++l)
            for (int s = 0; s < m; ++s) qr[l * m + s] = pi[s];
        qe[(size_t)t.root * P + p] = 0;
    }
    for (int o = 0; o < n; ++o) {
        int k = t.order[o];
        if (k < n_tips) continue;
        for (int oi = t.kid_off[k]; oi < t.kid_off[k + 1]; ++oi) {
            int ci = t.kids[oi];   /* child being updated; every other child of k is a sibling */
            for (int p = 0; p < P; ++p) {
                const double *qk = pre + ((size_t)k * P + p) * row;
                double *qi = pre + ((size_t)ci * P + p) * row;
                int es = 0;
                for (int l = 0; l < C; ++l) {
                    /* u = q_k o (product over the siblings s of P_s p_s) */
                    for (int s2 = 0; s2 < m; ++s2) u[s2] = qk[l * m + s2];
                    for (int oj = t.kid_off[k]; oj < t.kid_off[k + 1]; ++oj) {
                        int cj = t.kids[oj];
                        if (cj == ci) continue;
                        const double *pj_ = post + ((size_t)cj * P + p) * row;
                        const double *Pj = Pm + ((size_t)cj * C + l) * mm;
                        for (int s2 = 0; s2 < m; ++s2) {
                            double a = 0.0;
                            for (int x = 0; x < m; ++x) a += Pj[s2 * m + x] * pj_[l * m + x];
                            u[s2] *= a;
                        }
                    }
                    const double *Pi = Pm + ((size_t)ci * C + l) * mm;
                    for (int x = 0; x < m; ++x) {
                        double a = 0.0;
                        for (int s2 = 0; s2 < m; ++s2) a += Pi[s2 * m + x] * u[s2];
                        qi[l * m + x] = a;
                    }
                }
                for (int oj = t.kid_off[k]; oj < t.kid_off[k + 1]; ++oj)
                    if (t.kids[oj] != ci) es += pe[(size_t)t.kids[oj] * P + p];
                qe[(size_t)ci * P + p] = qe[(size_t)k * P + p] + es + rescale(qi, (int)row);
            }
        }
    }

    /* gradient and Hessian diagonal: for branch i,
     *   g_p = sum_l r_l w_l p_i,l' Q_i' q_i,l / L_p,   h_p = sum_l r_l^2 w_l p' (Q_i^2)' q / L_p - g_p^2 */
    for (int i = 0; i < n; ++i) {
        double gsum = 0.0, hsum = 0.0;
        if (i != t.root) {
            const double *Qi = Q + (size_t)(branch_model ? branch_model[i] : 0) * mm;
            mat_mul(m, Qi, Qi, Q2);
            for (int p = 0; p < P; ++p) {
                const double *pp = post + ((size_t)i * P + p) * row;
                const double *qq = pre + ((size_t)i * P + p) * row;
                double g = 0.0, h = 0.0;
                for (int l = 0; l < C; ++l) {
                    double d1 = 0.0, d2 = 0.0;   /* p' Q' q = q' Q p ;  p' (Q^2)' q */
                    for (int s = 0; s < m; ++s)
                        for (int x = 0; x < m; ++x) {
                            d1 += qq[l * m + s] * Qi[s * m + x] * pp[l * m + x];
                            d2 += qq[l * m + s] * Q2[s * m + x] * pp[l * m + x];
                        }
                    g += rates[l] * cat_w[l] * d1;
                    h += rates[l] * rates[l] * cat_w[l] * d2;
                }
                int ex = pe[(size_t)i * P + p] + qe[(size_t)i * P + p] - pe[(size_t)t.root * P + p];
                double gp = ldexp(g, ex) / Lhat[p];
                double hp = ldexp(h, ex) / Lhat[p] - gp * gp;
                gsum += weights[p] * gp;
                hsum += weights[p] * hp;
            }
        }
        if (grad) grad[i] = gsum;
        if (hess) hess[i] = hsum;
    }

    if (post_out) memcpy(post_out, post, (size_t)n * P * row * sizeof(double));
    if (pre_out) memcpy(pre_out, pre, (size_t)n * P * row * sizeof(double));
    if (post_e_out) memcpy(post_e_out, pe, (size_t)n * P * sizeof(int32_t));
    if (pre_e_out) memcpy(pre_e_out, qe, (size_t)n * P * sizeof(int32_t));
    rc = ORC_OK;
done:
    free(Pm); free(post); free(pre); free(pe); free(qe); free(Lhat);
    free(A); free(Q2); free(u);
    tree_free(&t);
    return rc;
}

/* The paper's binary tree: n_nodes = 2 n_tips - 1. */
int orc_eval(int n_tips, int m, int n_patterns, int n_cat, int n_models,
             const int32_t *parent, const uint8_t *tips, const double *weights,
             const double *Q, const int32_t *branch_model, const double *pi,
             const double *rates, const double *cat_w, const double *b,
             int n_tip_vecs, const double *tip_vecs,
             double *logL, double *grad, double *site_logL, double *hess,
             double *post_out, double *pre_out, int32_t *post_e_out, int32_t *pre_e_out)
{
    return orc_eval_tree(n_tips, 2 * n_tips - 1, m, n_patterns, n_cat, n_models, parent, tips, weights, Q,
                         branch_model, pi, rates, cat_w, b, n_tip_vecs, tip_vecs, logL, grad, site_logL, hess,
                         post_out, pre_out, post_e_out, pre_e_out);
}
