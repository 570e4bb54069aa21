/*
 * SGD_Tucker FP64 reference oracle (Li et al., arXiv 2012.03550).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline / reference legs may load it.  It
 * shares no code, header, table or helper with the CUDA library, and it never
 * reads anything the CUDA path produced.
 *
 * Everything is FP64 (the paper runs all experiments in double precision,
 * Sec. 5.1).  Indices are 0-based (the paper is 1-based).
 *
 * Notation follows the paper:
 *   N order, I_n mode sizes, J_n ranks, R = R_core Kruskal rank of the core,
 *   A(n) in R^{I_n x J_n} factor matrices (row-major, row i = a^(n)_{i,:}),
 *   B(n) in R^{J_n x R} Kruskal matrices of the core (row-major, column r = b^(n)_{:,r}),
 *   G-hat the core built from B by Eq. 4, stored mode-1-fastest:
 *       lin(j_1..j_N) = j_1 + J_1*(j_2 + J_2*(j_3 + ...)).
 *   Mode-n unfolding (Def. 1): column c of G_(n) enumerates (j_k)_{k != n}
 *   with the lowest remaining mode fastest, c = sum_{k!=n} j_k prod_{m<k,m!=n} J_m.
 *   The Kronecker row S_s of a sample (Eq. 10, S = A(N) x ... x A(n+1) x
 *   A(n-1) x ... x A(1)) uses the same column order: S_s[c] = prod_{k!=n} a_k[j_k(c)].
 *   Vectorisation (Def. 2): element (row j, column c) of G_(n) sits at c*J_n + j.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   - gradients are used exactly as printed in Eq. 15 and Eq. 18 (no factor 2);
 *   - SGD(M, lambda, gamma, w, grad) of Sec. 3.2 / Eq. 3 is
 *       w <- w - gamma * (grad / M + lambda * w);
 *   - the factor-row normaliser is the minibatch size M (Eq. 18) by default;
 *     norm_mode 1 uses |Psi_i| (Algorithm 1, factor update line);
 *   - an epoch is one pass over a keyed pseudorandom permutation of the
 *     training entries in consecutive chunks of M; the last chunk uses its
 *     own size as M;
 *   - within one factor phase every row reads the state before that phase's
 *     updates of the same mode (rows are independent, Eq. 12); across modes
 *     and across r_core the updates are sequential (Algorithm 1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAXN 8

/* Error codes (mirroring no other file on purpose). */
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* Minibatch sampler.                                                        */
/*                                                                            */
/* The paper draws the M-entry set Psi at random from Omega (Sec. 3.2, Eq. 3; */
/* input of Algorithm 1).  Reading: epoch e visits the training entries in    */
/* the order of a keyed pseudorandom permutation pi_e of [0, n), minibatch b  */
/* being positions [bM, bM+M).  pi_e is a balanced Feistel network (Luby &    */
/* Rackoff 1988) on 2h bits, 2h the smallest even width with 2^(2h) >= n      */
/* (h >= 1), restricted to [0, n) by cycle walking (Black & Rogaway 2002).    */
/* Six rounds; round i maps (L, R) -> (R, L xor (F(R xor K_i) & (2^h - 1))),  */
/* x = L * 2^h + R, with F the SplitMix64 output function (Steele, Lea &      */
/* Flood 2014) and K_i = F(seed + (8*epoch + i + 1) * 0x9E3779B97F4A7C15).    */
/* ------------------------------------------------------------------------ */
static uint64_t orc_splitmix_out(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int orc_half_bits(uint64_t n)
{
    int b = 0;
    while (b < 64 && (n - 1) >> b) /* bits needed for n-1 */
        b++;
    if (n <= 1) b = 0;
    int h = (b + 1) / 2;
    return h < 1 ? 1 : h;
}

static uint64_t orc_feistel(uint64_t x, int h, const uint64_t key[6])
{
    uint64_t mask = (h >= 64) ? ~0ULL : ((1ULL << h) - 1ULL);
    uint64_t L = x >> h, R = x & mask;
    for (int i = 0; i < 6; ++i) {
        uint64_t f = orc_splitmix_out(R ^ key[i]) & mask;
        uint64_t nl = R;
        R = L ^ f;
        L = nl;
    }
    return (L << h) | R;
}

static void orc_round_keys(uint64_t seed, uint64_t epoch, uint64_t key[6])
{
    for (int i = 0; i < 6; ++i)
        key[i] = orc_splitmix_out(seed + (8ULL * epoch + (uint64_t)i + 1ULL) * 0x9E3779B97F4A7C15ULL);
}

/* pi_e(t) for one position t in [0, n). */
uint64_t orc_perm(uint64_t n, uint64_t seed, uint64_t epoch, uint64_t t)
{
    uint64_t key[6];
    orc_round_keys(seed, epoch, key);
    int h = orc_half_bits(n);
    uint64_t y = orc_feistel(t, h, key);
    while (y >= n)
        y = orc_feistel(y, h, key);
    return y;
}

/* pi_e(t) for t in [t0, t0+count). */
void orc_perm_range(uint64_t n, uint64_t seed, uint64_t epoch, int64_t t0, int64_t count, int64_t *out)
{
    for (int64_t q = 0; q < count; ++q)
        out[q] = (int64_t)orc_perm(n, seed, epoch, (uint64_t)(t0 + q));
}

/* ------------------------------------------------------------------------ */
/* Minibatch tiling by mode index.                                            */
/* The improved strategy of Sec. 4.4.2 keeps one COO copy and groups the      */
/* samples of Psi that share a row i_n of A(n) (Algorithm 1, factor loop over */
/* i_n).  Here: a stable sort of the batch positions by i_n, i.e. by the pair */
/* (i_n, position), and the boundaries of the runs of equal i_n (segments).   */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t key; int32_t pos; } orc_kp;

static int orc_kp_cmp(const void *a, const void *b)
{
    const orc_kp *x = (const orc_kp *)a, *y = (const orc_kp *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/* keys[m] -> order[m] (batch positions in sorted order), seg_off[U+1]
 * (segment start offsets into order, seg_off[U] = m).  Returns U. */
int64_t orc_stable_order(int64_t m, const int32_t *keys, int32_t *order, int32_t *seg_off)
{
    if (m <= 0) { if (seg_off) seg_off[0] = 0; return 0; }
    orc_kp *kp = (orc_kp *)malloc((size_t)m * sizeof(orc_kp));
    if (!kp) return -1;
    for (int64_t i = 0; i < m; ++i) { kp[i].key = keys[i]; kp[i].pos = (int32_t)i; }
    qsort(kp, (size_t)m, sizeof(orc_kp), orc_kp_cmp);
    int64_t u = 0;
    for (int64_t q = 0; q < m; ++q) {
        order[q] = kp[q].pos;
        if (q == 0 || kp[q].key != kp[q - 1].key) {
            if (seg_off) seg_off[u] = (int32_t)q;
            u++;
        }
    }
    if (seg_off) seg_off[u] = (int32_t)m;
    free(kp);
    return u;
}

/* ------------------------------------------------------------------------ */
/* Model.                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N, R;
    int64_t I[ORC_MAXN];
    int J[ORC_MAXN];
    double *A[ORC_MAXN];   /* I_n x J_n */
    double *B[ORC_MAXN];   /* J_n x R   */
    double *G;             /* prod J_n, mode-1 fastest */
} orc_model;

static int64_t orc_prodJ(const orc_model *md)
{
    int64_t p = 1;
    for (int n = 0; n < md->N; ++n) p *= md->J[n];
    return p;
}

/* Core from its Kruskal matrices, Eq. 4:
 *   G-hat = sum_r b^(1)_{:,r} o b^(2)_{:,r} o ... o b^(N)_{:,r}. */
static void orc_core_from_B(orc_model *md)
{
    int64_t P = orc_prodJ(md);
    int j[ORC_MAXN];
    for (int64_t lin = 0; lin < P; ++lin) {
        int64_t t = lin;
        for (int n = 0; n < md->N; ++n) { j[n] = (int)(t % md->J[n]); t /= md->J[n]; }
        double g = 0.0;
        for (int r = 0; r < md->R; ++r) {
            double prod = 1.0;
            for (int n = 0; n < md->N; ++n) prod *= md->B[n][(int64_t)j[n] * md->R + r];
            g += prod;
        }
        md->G[lin] = g;
    }
}

/* x-hat at one coordinate by the definition of the Tucker model (Def. 6):
 *   x-hat = sum_{j_1..j_N} G-hat[j] prod_n A(n)[i_n, j_n]. */
static double orc_predict_one(const orc_model *md, const int32_t *coord)
{
    int64_t P = orc_prodJ(md);
    int j[ORC_MAXN];
    double acc = 0.0;
    for (int64_t lin = 0; lin < P; ++lin) {
        int64_t t = lin;
        double prod = md->G[lin];
        for (int n = 0; n < md->N; ++n) {
            j[n] = (int)(t % md->J[n]); t /= md->J[n];
            prod *= md->A[n][(int64_t)coord[n] * md->J[n] + j[n]];
        }
        acc += prod;
    }
    return acc;
}

/* Column c of the mode-n unfolding (Def. 1) -> the digits (j_k)_{k != n}. */
static void orc_unfold_digits(const orc_model *md, int n, int64_t c, int *j)
{
    for (int k = 0; k < md->N; ++k) {
        if (k == n) continue;
        j[k] = (int)(c % md->J[k]);
        c /= md->J[k];
    }
}

/* Column of a full index in the mode-n unfolding of a tensor with dimensions
 * dims (Def. 1, 0-based): the inverse of orc_unfold_digits, written out from
 * the definition c = sum_{k != n} i_k prod_{m < k, m != n} dims_m. */
int64_t orc_unfold_column(int N, const int64_t *dims, int n, const int64_t *index)
{
    int64_t c = 0;
    for (int k = 0; k < N; ++k) {
        if (k == n) continue;
        int64_t stride = 1;
        for (int m = 0; m < k; ++m)
            if (m != n) stride *= dims[m];
        c += index[k] * stride;
    }
    return c;
}

/* Public wrapper of orc_unfold_digits for the convention pin. */
void orc_unfold_digits_public(int N, const int32_t *J, int n, int64_t c, int32_t *digits)
{
    orc_model md;
    memset(&md, 0, sizeof(md));
    md.N = N;
    for (int k = 0; k < N; ++k) md.J[k] = J[k];
    int j[ORC_MAXN] = {0};
    orc_unfold_digits(&md, n, c, j);
    for (int k = 0; k < N; ++k) digits[k] = (k == n) ? -1 : j[k];
}

static int64_t orc_lin(const orc_model *md, const int *j)
{
    int64_t lin = 0, stride = 1;
    for (int k = 0; k < md->N; ++k) { lin += (int64_t)j[k] * stride; stride *= md->J[k]; }
    return lin;
}

/* ------------------------------------------------------------------------ */
/* Core phase of Algorithm 1 for one mode n.                                  */
/*                                                                            */
/* W_r (M x J_n) = H_Psi O_r.  Literal form: H_Psi row s is                   */
/* Vec_n of the outer product of the sample's factor rows (Eq. 5, Def. 2:     */
/* H_s[c*J_n + j] = a_n[j] * S_s[c]); O_r stacks q_{c,r} U (Eq. 7) with       */
/* Q(n) = B(N) (.) ... (.) B(n+1) (.) B(n-1) (.) ... (.) B(1) (Eq. 5).        */
/* Closed form used at scale (the same numbers by the mixed-product property  */
/* of the Kronecker product): W_r[s][j] = a_n[j] * prod_{k!=n} <a_k, b^(k)_r>. */
/* ------------------------------------------------------------------------ */
static int orc_build_W(const orc_model *md, int n, int64_t m, const int32_t *coords,
                       int literal, double *W /* R x m x J_n */)
{
    const int N = md->N, R = md->R, Jn = md->J[n];
    if (!literal) {
        for (int r = 0; r < R; ++r)
            for (int64_t s = 0; s < m; ++s) {
                const int32_t *co = coords + s * N;
                double w = 1.0;
                for (int k = 0; k < N; ++k) {
                    if (k == n) continue;
                    const double *a = md->A[k] + (int64_t)co[k] * md->J[k];
                    double dot = 0.0;
                    for (int j = 0; j < md->J[k]; ++j) dot += a[j] * md->B[k][(int64_t)j * R + r];
                    w *= dot;
                }
                const double *an = md->A[n] + (int64_t)co[n] * Jn;
                for (int j = 0; j < Jn; ++j) W[((int64_t)r * m + s) * Jn + j] = an[j] * w;
            }
        return ORC_OK;
    }
    /* Literal: H (m x prodJ), Q (P_n x R), O_r (prodJ x J_n), W_r = H O_r. */
    const int64_t P = orc_prodJ(md);
    const int64_t Pn = P / Jn;
    double *H = (double *)malloc((size_t)(m * P) * sizeof(double));
    double *Q = (double *)malloc((size_t)(Pn * R) * sizeof(double));
    double *O = (double *)malloc((size_t)(P * Jn) * sizeof(double));
    if (!H || !Q || !O) { free(H); free(Q); free(O); return ORC_ENOMEM; }
    int jd[ORC_MAXN];
    for (int64_t s = 0; s < m; ++s) {           /* H_Psi */
        const int32_t *co = coords + s * N;
        for (int64_t c = 0; c < Pn; ++c) {
            orc_unfold_digits(md, n, c, jd);
            double Sc = 1.0;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                Sc *= md->A[k][(int64_t)co[k] * md->J[k] + jd[k]];
            }
            for (int j = 0; j < Jn; ++j)
                H[s * P + c * Jn + j] = md->A[n][(int64_t)co[n] * Jn + j] * Sc;
        }
    }
    for (int64_t c = 0; c < Pn; ++c) {          /* Q(n), Khatri-Rao of the other B */
        orc_unfold_digits(md, n, c, jd);
        for (int r = 0; r < R; ++r) {
            double q = 1.0;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                q *= md->B[k][(int64_t)jd[k] * R + r];
            }
            Q[c * R + r] = q;
        }
    }
    for (int r = 0; r < R; ++r) {               /* W_r for every column r */
        memset(O, 0, (size_t)(P * Jn) * sizeof(double));   /* O_r by Eq. 7 */
        for (int64_t c = 0; c < Pn; ++c)
            for (int j = 0; j < Jn; ++j) O[(c * Jn + j) * Jn + j] = Q[c * R + r];
        for (int64_t s = 0; s < m; ++s)          /* W_r = H_Psi O_r */
            for (int j = 0; j < Jn; ++j) {
                double acc = 0.0;
                for (int64_t k = 0; k < P; ++k) acc += H[s * P + k] * O[k * Jn + j];
                W[((int64_t)r * m + s) * Jn + j] = acc;
            }
    }
    free(H); free(Q); free(O);
    return ORC_OK;
}

/* V for block (n, rc) at the current B (Algorithm 1, core phase, Eq. 15):
 *   x-hat = x - sum_{r != rc} W_r b_r;  C = W_rc^T W_rc;  V = -W_rc^T x-hat + C b_rc.
 * This V is the bracket of Eq. 15, i.e. grad = V / M + lambda_B b_rc. */
static void orc_core_V(const orc_model *md, int n, int rc, int64_t m, const double *x,
                       const double *W, double *xhat, double *C, double *V)
{
    const int R = md->R, Jn = md->J[n];
    for (int64_t s = 0; s < m; ++s) xhat[s] = x[s];                      /* x-hat starts at x */
    for (int r = 0; r < R; ++r) {                                          /* minus the other columns */
        if (r == rc) continue;
        for (int64_t s = 0; s < m; ++s) {
            double wb = 0.0;
            for (int j = 0; j < Jn; ++j)
                wb += W[((int64_t)r * m + s) * Jn + j] * md->B[n][(int64_t)j * R + r];
            xhat[s] -= wb;
        }
    }
    for (int a = 0; a < Jn; ++a)                                           /* Gram W_rc^T W_rc */
        for (int b = 0; b < Jn; ++b) {
            double acc = 0.0;
            for (int64_t s = 0; s < m; ++s)
                acc += W[((int64_t)rc * m + s) * Jn + a] * W[((int64_t)rc * m + s) * Jn + b];
            C[a * Jn + b] = acc;
        }
    for (int a = 0; a < Jn; ++a) {                                         /* V */
        double acc = 0.0;
        for (int64_t s = 0; s < m; ++s) acc -= W[((int64_t)rc * m + s) * Jn + a] * xhat[s];
        for (int b = 0; b < Jn; ++b) acc += C[a * Jn + b] * md->B[n][(int64_t)b * R + rc];
        V[a] = acc;
    }
}

/* SGD(M, lambda, gamma, w, grad) (Sec. 3.2, Eq. 3): w <- w - gamma (grad/M + lambda w),
 * returned as the change delta = -(gamma (grad/M + lambda w)); the caller sets
 * w <- w + delta, which is the same IEEE result as w - gamma (...) (x - y is
 * x + (-y) exactly, and this file is compiled without contraction). */
static double orc_sgd_delta(double w, double grad, double M, double lambda, double gamma)
{
    return -(gamma * (grad / M + lambda * w));
}

/* Heavy-ball momentum (Polyak 1964), the accelerated SGD the paper names as
 * future work (Sec. 6): with g = grad / M + lambda w the velocity becomes
 * v <- mu v + g and the parameter w <- w - gamma v (returned as the change
 * -(gamma v)).  mu = 0 gives orc_sgd_delta. */
static double orc_sgd_momentum_delta(double w, double *v, double grad, double M, double lambda, double gamma,
                                     double mu)
{
    const double g = grad / M + lambda * w;
    *v = mu * (*v) + g;
    return -(gamma * (*v));
}

/* ------------------------------------------------------------------------ */
/* Factor phase of Algorithm 1 for one mode n and one row i_n                */
/* whose samples are sample_ids[0..cnt).                                     */
/*   S rows (Eq. 10), E = G_(n) S^T (Eq. 11),                                 */
/*   C = E E^T, F = -X E^T + a C.                                             */
/* F is the bracket of Eq. 18, i.e. grad = F / M + lambda_A a.                */
/* ------------------------------------------------------------------------ */
static void orc_factor_F(const orc_model *md, int n, const int32_t *coords, const double *x,
                         const int32_t *sample_ids, int64_t cnt, double *E /* cnt x J_n */,
                         double *C /* J_n x J_n */, double *F /* J_n */)
{
    const int N = md->N, Jn = md->J[n];
    const int64_t Pn = orc_prodJ(md) / Jn;
    int jd[ORC_MAXN];
    for (int64_t q = 0; q < cnt; ++q) {
        const int32_t *co = coords + (int64_t)sample_ids[q] * N;
        for (int j = 0; j < Jn; ++j) E[q * Jn + j] = 0.0;
        for (int64_t c = 0; c < Pn; ++c) {
            orc_unfold_digits(md, n, c, jd);
            double Sc = 1.0;                                        /* S (Eq. 10) */
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                Sc *= md->A[k][(int64_t)co[k] * md->J[k] + jd[k]];
            }
            for (int j = 0; j < Jn; ++j) {                           /* E (Eq. 11) */
                jd[n] = j;
                E[q * Jn + j] += md->G[orc_lin(md, jd)] * Sc;
            }
        }
    }
    for (int a = 0; a < Jn; ++a)                                     /* C = E E^T */
        for (int b = 0; b < Jn; ++b) {
            double acc = 0.0;
            for (int64_t q = 0; q < cnt; ++q) acc += E[q * Jn + a] * E[q * Jn + b];
            C[a * Jn + b] = acc;
        }
    const int32_t *co0 = coords + (int64_t)sample_ids[0] * N;
    const double *ai = md->A[n] + (int64_t)co0[n] * Jn;
    for (int b = 0; b < Jn; ++b) {                                   /* F */
        double acc = 0.0;
        for (int64_t q = 0; q < cnt; ++q) acc -= x[sample_ids[q]] * E[q * Jn + b];
        for (int a = 0; a < Jn; ++a) acc += ai[a] * C[a * Jn + b];
        F[b] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Exported API (ctypes).                                                     */
/* ------------------------------------------------------------------------ */
static int orc_setup(orc_model *md, int N, const int64_t *I, const int32_t *J, int R,
                     double **A, double **B, double *G)
{
    if (N < 1 || N > ORC_MAXN || R < 1) return ORC_EINVAL;
    md->N = N; md->R = R;
    for (int n = 0; n < N; ++n) {
        if (J[n] < 1 || I[n] < 1) return ORC_EINVAL;
        md->I[n] = I[n]; md->J[n] = J[n]; md->A[n] = A[n]; md->B[n] = B[n];
    }
    md->G = G;
    return ORC_OK;
}

/* G-hat from B (Eq. 4). */
int orc_build_core(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G)
{
    orc_model md;
    int rc = orc_setup(&md, N, I, J, R, A, B, G);
    if (rc) return rc;
    orc_core_from_B(&md);
    return ORC_OK;
}

/* x-hat at k coordinates (Def. 6) with G-hat built from B (Eq. 4). */
int orc_predict(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                int64_t k, const int32_t *coords, double *out)
{
    orc_model md;
    int rc = orc_setup(&md, N, I, J, R, A, B, G);
    if (rc) return rc;
    orc_core_from_B(&md);
    for (int64_t s = 0; s < k; ++s) out[s] = orc_predict_one(&md, coords + s * N);
    return ORC_OK;
}

/* RMSE and MAE over k entries (Eq. 19). */
int orc_rmse_mae(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                 int64_t k, const int32_t *coords, const float *values, double *rmse, double *mae)
{
    orc_model md;
    int rc = orc_setup(&md, N, I, J, R, A, B, G);
    if (rc) return rc;
    orc_core_from_B(&md);
    double se = 0.0, ae = 0.0;
    for (int64_t s = 0; s < k; ++s) {
        double d = (double)values[s] - orc_predict_one(&md, coords + s * N);
        se += d * d;
        ae += fabs(d);
    }
    *rmse = k > 0 ? sqrt(se / (double)k) : 0.0;
    if (mae) *mae = k > 0 ? ae / (double)k : 0.0;
    return ORC_OK;
}

/* Eq. 15 gradient of block b^(n)_{:,r} at the current state for the m samples
 * coords/x (no update): out = V / m + lambda_B b_r. */
int orc_core_gradient(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B,
                      int64_t m, const int32_t *coords, const float *values, int n, int r,
                      double lambda_b, int literal, double *out)
{
    orc_model md;
    int rc = orc_setup(&md, N, I, J, R, A, B, NULL);
    if (rc) return rc;
    if (n < 0 || n >= N || r < 0 || r >= R || m < 1) return ORC_EINVAL;
    const int Jn = md.J[n];
    double *W = (double *)malloc((size_t)(R * m * Jn) * sizeof(double));
    double *x = (double *)malloc((size_t)m * sizeof(double));
    double *xh = (double *)malloc((size_t)m * sizeof(double));
    double *C = (double *)malloc((size_t)(Jn * Jn) * sizeof(double));
    double *V = (double *)malloc((size_t)Jn * sizeof(double));
    if (!W || !x || !xh || !C || !V) { free(W); free(x); free(xh); free(C); free(V); return ORC_ENOMEM; }
    for (int64_t s = 0; s < m; ++s) x[s] = values[s];
    rc = orc_build_W(&md, n, m, coords, literal, W);
    if (!rc) {
        orc_core_V(&md, n, r, m, x, W, xh, C, V);
        for (int j = 0; j < Jn; ++j) out[j] = V[j] / (double)m + lambda_b * md.B[n][(int64_t)j * R + r];
    }
    free(W); free(x); free(xh); free(C); free(V);
    return rc;
}

/* Eq. 18 gradient of row a^(n)_{row,:} at the current state over the samples
 * of coords/x whose mode-n index is `row`: out = F / denom + lambda_A a. */
int orc_factor_gradient(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B,
                        double *G, int64_t m, const int32_t *coords, const float *values, int n,
                        int32_t row, double lambda_a, int norm_mode, double *out)
{
    orc_model md;
    int rc = orc_setup(&md, N, I, J, R, A, B, G);
    if (rc) return rc;
    if (n < 0 || n >= N || m < 1) return ORC_EINVAL;
    orc_core_from_B(&md);
    const int Jn = md.J[n];
    int32_t *ids = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    double *x = (double *)malloc((size_t)m * sizeof(double));
    double *E = (double *)malloc((size_t)(m * Jn) * sizeof(double));
    double *C = (double *)malloc((size_t)(Jn * Jn) * sizeof(double));
    double *F = (double *)malloc((size_t)Jn * sizeof(double));
    if (!ids || !x || !E || !C || !F) { free(ids); free(x); free(E); free(C); free(F); return ORC_ENOMEM; }
    int64_t cnt = 0;
    for (int64_t s = 0; s < m; ++s) {
        x[s] = values[s];
        if (coords[s * N + n] == row) ids[cnt++] = (int32_t)s;
    }
    if (cnt == 0) {
        for (int j = 0; j < Jn; ++j) out[j] = 0.0;
    } else {
        orc_factor_F(&md, n, coords, x, ids, cnt, E, C, F);
        double denom = norm_mode == 1 ? (double)cnt : (double)m;
        const double *a = md.A[n] + (int64_t)row * Jn;
        for (int j = 0; j < Jn; ++j) out[j] = F[j] / denom + lambda_a * a[j];
    }
    free(ids); free(x); free(E); free(C); free(F);
    return ORC_OK;
}

/*
 * One SGD_Tucker minibatch step, Algorithm 1, on the m samples coords/values
 * (in minibatch order).  Updates A and B in place and leaves G-hat built from
 * the new B.  If probe_V is non-NULL it receives, for every mode n and r_core,
 * the core-phase bracket V of Eq. 15 (layout [n][r][Jmax]); if probe_F is non-NULL it
 * receives, for every mode n and every segment u of equal i_n in ascending
 * i_n, the factor-phase bracket F of Eq. 18 (layout [n][u][Jmax], u < m), with the number of
 * segments per mode in probe_nseg[n].
 */
static int orc_step_impl(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                         int64_t m, const int32_t *coords, const float *values,
                         double gamma_a, double gamma_b, double lambda_a, double lambda_b,
                         int norm_mode, int literal, double *probe_V, double *probe_F, int64_t *probe_nseg,
                         double mu, double **VA, double **VB, double **accA, double **accB);

int orc_step_momentum(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                      int64_t m, const int32_t *coords, const float *values,
                      double gamma_a, double gamma_b, double lambda_a, double lambda_b,
                      int norm_mode, int literal, double *probe_V, double *probe_F, int64_t *probe_nseg,
                      double mu, double **VA, double **VB);

int orc_step(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
             int64_t m, const int32_t *coords, const float *values,
             double gamma_a, double gamma_b, double lambda_a, double lambda_b,
             int norm_mode, int literal, double *probe_V, double *probe_F, int64_t *probe_nseg)
{
    return orc_step_momentum(N, I, J, R, A, B, G, m, coords, values, gamma_a, gamma_b, lambda_a, lambda_b,
                             norm_mode, literal, probe_V, probe_F, probe_nseg, 0.0, NULL, NULL);
}

/*
 * orc_step with heavy-ball momentum: VA[n] (I_n x J_n) and VB[n] (J_n x R)
 * hold the velocities of the factor rows and of the Kruskal columns; every
 * update of Algorithm 1 (Kruskal columns and factor rows) goes through orc_sgd_momentum.  A row
 * untouched by the minibatch keeps its velocity (as it keeps its value).
 * VA = VB = NULL gives plain SGD.
 */
int orc_step_momentum(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                      int64_t m, const int32_t *coords, const float *values,
                      double gamma_a, double gamma_b, double lambda_a, double lambda_b,
                      int norm_mode, int literal, double *probe_V, double *probe_F, int64_t *probe_nseg,
                      double mu, double **VA, double **VB)
{
    return orc_step_impl(N, I, J, R, A, B, G, m, coords, values, gamma_a, gamma_b, lambda_a, lambda_b, norm_mode,
                         literal, probe_V, probe_F, probe_nseg, mu, VA, VB, NULL, NULL);
}

/*
 * The step itself.  Every update w <- w + delta of Algorithm 1 is applied to
 * the model (A, B), which this minibatch's own later steps read (Gauss-Seidel
 * order); when accA / accB are given, the same delta is also added to the
 * matching entry of a second model (accA[n] like A[n], accB[n] like B[n]):
 * the accumulation of the K-snapshot form (orc_epoch_snapshot).
 */
static int orc_step_impl(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                         int64_t m, const int32_t *coords, const float *values,
                         double gamma_a, double gamma_b, double lambda_a, double lambda_b,
                         int norm_mode, int literal, double *probe_V, double *probe_F, int64_t *probe_nseg,
                         double mu, double **VA, double **VB, double **accA, double **accB)
{
    orc_model md;
    int rc = orc_setup(&md, N, I, J, R, A, B, G);
    if (rc) return rc;
    if (m < 1) return ORC_EINVAL;
    int Jmax = 0;
    for (int n = 0; n < N; ++n) if (md.J[n] > Jmax) Jmax = md.J[n];
    double *x = (double *)malloc((size_t)m * sizeof(double));
    double *W = (double *)malloc((size_t)(R * m * Jmax) * sizeof(double));
    double *xh = (double *)malloc((size_t)m * sizeof(double));
    double *C = (double *)malloc((size_t)(Jmax * Jmax) * sizeof(double));
    double *V = (double *)malloc((size_t)Jmax * sizeof(double));
    double *E = (double *)malloc((size_t)(m * Jmax) * sizeof(double));
    double *F = (double *)malloc((size_t)Jmax * sizeof(double));
    int32_t *keys = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *seg = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    if (!x || !W || !xh || !C || !V || !E || !F || !keys || !order || !seg) { rc = ORC_ENOMEM; goto done; }
    for (int64_t s = 0; s < m; ++s) x[s] = values[s];

    /* Core phase. */
    for (int n = 0; n < N; ++n) {
        const int Jn = md.J[n];
        rc = orc_build_W(&md, n, m, coords, literal, W);             /* W_r, Eq. 7 */
        if (rc) goto done;
        for (int r = 0; r < R; ++r) {                                 /* cyclic over r */
            orc_core_V(&md, n, r, m, x, W, xh, C, V);
            if (probe_V)
                for (int j = 0; j < Jn; ++j) probe_V[((int64_t)n * R + r) * Jmax + j] = V[j];
            for (int j = 0; j < Jn; ++j) {                            /* b_r update */
                double *b = &md.B[n][(int64_t)j * R + r];
                double d;
                if (VB)
                    d = orc_sgd_momentum_delta(*b, &VB[n][(int64_t)j * R + r], V[j], (double)m, lambda_b,
                                               gamma_b, mu);
                else
                    d = orc_sgd_delta(*b, V[j], (double)m, lambda_b, gamma_b);
                *b = *b + d;
                if (accB) accB[n][(int64_t)j * R + r] += d;
            }
        }
    }
    orc_core_from_B(&md);                                             /* Eq. 4 */

    /* Factor phase. */
    for (int n = 0; n < N; ++n) {
        const int Jn = md.J[n];
        for (int64_t s = 0; s < m; ++s) keys[s] = coords[s * N + n];
        int64_t U = orc_stable_order(m, keys, order, seg);
        if (U < 0) { rc = ORC_ENOMEM; goto done; }
        if (probe_nseg) probe_nseg[n] = U;
        for (int64_t u = 0; u < U; ++u) {                             /* each touched row */
            int64_t cnt = seg[u + 1] - seg[u];
            const int32_t *ids = order + seg[u];
            orc_factor_F(&md, n, coords, x, ids, cnt, E, C, F);
            if (probe_F)
                for (int j = 0; j < Jn; ++j) probe_F[((int64_t)n * m + u) * Jmax + j] = F[j];
            double denom = norm_mode == 1 ? (double)cnt : (double)m;
            const int64_t row = coords[(int64_t)ids[0] * N + n];
            double *a = md.A[n] + row * Jn;
            for (int j = 0; j < Jn; ++j) {                            /* row update */
                double d;
                if (VA)
                    d = orc_sgd_momentum_delta(a[j], &VA[n][row * Jn + j], F[j], denom, lambda_a, gamma_a, mu);
                else
                    d = orc_sgd_delta(a[j], F[j], denom, lambda_a, gamma_a);
                a[j] = a[j] + d;
                if (accA) accA[n][row * Jn + j] += d;
            }
        }
    }
done:
    free(x); free(W); free(xh); free(C); free(V); free(E); free(F); free(keys); free(order); free(seg);
    return rc;
}

/*
 * Minibatches [batch_begin, batch_end) of epoch `epoch` over the n_train
 * training entries (coords n_train x N, values n_train): minibatch b is the
 * entries pi_e(t), t in [bM, min(bM+M, n_train)).
 */
int orc_epoch_momentum(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                       int64_t n_train, const int32_t *coords, const float *values, int64_t M,
                       uint64_t seed, uint64_t epoch, int64_t batch_begin, int64_t batch_end,
                       double gamma_a, double gamma_b, double lambda_a, double lambda_b, int norm_mode,
                       double mu, double **VA, double **VB);

int orc_epoch(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
              int64_t n_train, const int32_t *coords, const float *values, int64_t M,
              uint64_t seed, uint64_t epoch, int64_t batch_begin, int64_t batch_end,
              double gamma_a, double gamma_b, double lambda_a, double lambda_b, int norm_mode)
{
    return orc_epoch_momentum(N, I, J, R, A, B, G, n_train, coords, values, M, seed, epoch, batch_begin,
                              batch_end, gamma_a, gamma_b, lambda_a, lambda_b, norm_mode, 0.0, NULL, NULL);
}

/* orc_epoch with heavy-ball momentum (velocities VA, VB as in orc_step_momentum). */
int orc_epoch_momentum(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                       int64_t n_train, const int32_t *coords, const float *values, int64_t M,
                       uint64_t seed, uint64_t epoch, int64_t batch_begin, int64_t batch_end,
                       double gamma_a, double gamma_b, double lambda_a, double lambda_b, int norm_mode,
                       double mu, double **VA, double **VB)
{
    if (M < 1 || n_train < 1 || N < 1 || N > ORC_MAXN) return ORC_EINVAL;
    int64_t nb = (n_train + M - 1) / M;
    if (batch_begin < 0) batch_begin = 0;
    if (batch_end > nb) batch_end = nb;
    int32_t *bc = (int32_t *)malloc((size_t)(M * N) * sizeof(int32_t));
    float *bv = (float *)malloc((size_t)M * sizeof(float));
    if (!bc || !bv) { free(bc); free(bv); return ORC_ENOMEM; }
    uint64_t key[6];
    orc_round_keys(seed, epoch, key);
    int h = orc_half_bits((uint64_t)n_train);
    int rc = ORC_OK;
    for (int64_t b = batch_begin; b < batch_end && rc == ORC_OK; ++b) {
        int64_t t0 = b * M;
        int64_t m = (t0 + M <= n_train) ? M : n_train - t0;
        for (int64_t q = 0; q < m; ++q) {
            uint64_t y = orc_feistel((uint64_t)(t0 + q), h, key);
            while (y >= (uint64_t)n_train) y = orc_feistel(y, h, key);
            for (int n = 0; n < N; ++n) bc[q * N + n] = coords[(int64_t)y * N + n];
            bv[q] = values[y];
        }
        rc = orc_step_momentum(N, I, J, R, A, B, G, m, bc, bv, gamma_a, gamma_b, lambda_a, lambda_b,
                               norm_mode, 0, NULL, NULL, NULL, mu, VA, VB);
    }
    free(bc); free(bv);
    return rc;
}

/*
 * K-snapshot form of the minibatch sequence (not Algorithm 1's order: a
 * labelled variant).  The minibatches [batch_begin, batch_end) of epoch
 * `epoch` are taken in blocks of K consecutive ones, the first block starting
 * at batch_begin.  Every minibatch of a block runs Algorithm 1's step (core
 * phase, G-hat, factor phase, with its own Gauss-Seidel order) from the same
 * snapshot: the model as it stood when the block began.  The changes delta
 * each minibatch made to the Kruskal columns and factor rows are then added
 * to the snapshot in minibatch order:
 *     theta <- ((theta_0 + delta_1) + delta_2) + ... + delta_K.
 * K = 1 is orc_epoch exactly (theta_0 + delta_1 is the strict step's
 * result).  Heavy-ball momentum is not defined for K > 1 (ORC_EINVAL).
 */
int orc_epoch_snapshot(int N, const int64_t *I, const int32_t *J, int R, double **A, double **B, double *G,
                       int64_t n_train, const int32_t *coords, const float *values, int64_t M,
                       uint64_t seed, uint64_t epoch, int64_t batch_begin, int64_t batch_end, int64_t K,
                       double gamma_a, double gamma_b, double lambda_a, double lambda_b, int norm_mode)
{
    if (M < 1 || n_train < 1 || N < 1 || N > ORC_MAXN || K < 1) return ORC_EINVAL;
    int64_t nb = (n_train + M - 1) / M;
    if (batch_begin < 0) batch_begin = 0;
    if (batch_end > nb) batch_end = nb;
    int32_t *bc = (int32_t *)malloc((size_t)(M * N) * sizeof(int32_t));
    float *bv = (float *)malloc((size_t)M * sizeof(float));
    double *WA[ORC_MAXN] = {0}, *WB[ORC_MAXN] = {0}, *SA[ORC_MAXN] = {0}, *SB[ORC_MAXN] = {0};
    int64_t P = 1;
    for (int n = 0; n < N; ++n) P *= J[n];
    double *WG = (double *)malloc((size_t)P * sizeof(double));
    int rc = (bc && bv && WG) ? ORC_OK : ORC_ENOMEM;
    for (int n = 0; n < N && rc == ORC_OK; ++n) {
        const size_t na = (size_t)I[n] * (size_t)J[n] * sizeof(double), nbb = (size_t)J[n] * R * sizeof(double);
        WA[n] = (double *)malloc(na); SA[n] = (double *)malloc(na);
        WB[n] = (double *)malloc(nbb); SB[n] = (double *)malloc(nbb);
        if (!WA[n] || !SA[n] || !WB[n] || !SB[n]) rc = ORC_ENOMEM;
    }
    uint64_t key[6];
    orc_round_keys(seed, epoch, key);
    int h = orc_half_bits((uint64_t)n_train);
    for (int64_t q0 = batch_begin; q0 < batch_end && rc == ORC_OK; q0 += K) {
        for (int n = 0; n < N; ++n) {                                   /* the snapshot theta_0 */
            memcpy(SA[n], A[n], (size_t)I[n] * J[n] * sizeof(double));
            memcpy(SB[n], B[n], (size_t)J[n] * R * sizeof(double));
        }
        for (int64_t b = q0; b < q0 + K && b < batch_end && rc == ORC_OK; ++b) {
            int64_t t0 = b * M;
            int64_t m = (t0 + M <= n_train) ? M : n_train - t0;
            for (int64_t q = 0; q < m; ++q) {
                uint64_t y = orc_feistel((uint64_t)(t0 + q), h, key);
                while (y >= (uint64_t)n_train) y = orc_feistel(y, h, key);
                for (int n = 0; n < N; ++n) bc[q * N + n] = coords[(int64_t)y * N + n];
                bv[q] = values[y];
            }
            for (int n = 0; n < N; ++n) {                               /* this minibatch starts at theta_0 */
                memcpy(WA[n], SA[n], (size_t)I[n] * J[n] * sizeof(double));
                memcpy(WB[n], SB[n], (size_t)J[n] * R * sizeof(double));
            }
            rc = orc_step_impl(N, I, J, R, WA, WB, WG, m, bc, bv, gamma_a, gamma_b, lambda_a, lambda_b,
                               norm_mode, 0, NULL, NULL, NULL, 0.0, NULL, NULL, A, B);
        }
    }
    if (rc == ORC_OK) {
        orc_model md;
        rc = orc_setup(&md, N, I, J, R, A, B, G);
        if (rc == ORC_OK) orc_core_from_B(&md);
    }
    for (int n = 0; n < N; ++n) { free(WA[n]); free(SA[n]); free(WB[n]); free(SB[n]); }
    free(WG); free(bc); free(bv);
    return rc;
}
