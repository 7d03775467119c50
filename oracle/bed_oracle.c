/*
 * bed_oracle.c -- FP64 CPU oracle for the batched divide-and-conquer symmetric
 * eigendecomposition of Y. Song, "A Short Note on Batch-efficient
 * Divide-and-Conquer Algorithm for EigenDecomposition" (arXiv 2604.27325).
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, sequential reference that
 * the CUDA path is checked against. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it; the library never does. It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Stages, in the paper's order (Sec. 2):
 *   a1  Householder tridiagonalization. Sec. 2 defers this stage to the
 *       authors' earlier work; it is written here as the textbook two-sided
 *       reduction (Golub & Van Loan, "Matrix Computations", Alg. 8.3.1).
 *   a2  Divide: rank-one tearing T = blkdiag(T1^, T2^) + |beta| v v^T,
 *       Eq. (1)-(3), recursively until the blocks are 2x2 (Sec. 2.1).
 *   a3  Leaves: one Givens/Jacobi rotation per 2x2 block (Sec. 2.2); with a
 *       larger leaf size, blocks of 3..8 rows by the implicit QL iteration with
 *       Wilkinson shifts (the "batched QR" leaf option the paper mentions,
 *       Sec. 2.2). The step recurrence is the published one of the EISPACK
 *       routine tql2 (Bowdler, Martin, Reinsch and Wilkinson, "The QR and QL
 *       algorithms for symmetric matrices", Numer. Math. 11, 1968), also given
 *       as tqli in Numerical Recipes; Golub & Van Loan Sec. 8.3 is the QR form.
 *   a4  Conquer: block spectral form Eq. (4) and coupling vector z Eq. (5);
 *       deflation (the paper does not describe it; Dongarra-Sorensen reading).
 *   a5  Secular equation Eq. (8) under the interlacing constraint Eq. (9)-(12):
 *       one bisection step Eq. (13)-(15), multi-section Eq. (16) until
 *       Eq. (17), then Halley's method Eq. (20)-(21) with the bracket kept
 *       by Eq. (14); roots are held as (nearer pole, offset) pairs.
 *   a6  Gu-Eisenstat recomputed z-hat Eq. (25) and normalized vectors Eq. (24).
 *   a7  Merge product Q = blkdiag(Q1, Q2) Q^ (Eq. (4)).
 *   a8  Back-transform V = H_0 H_1 ... H_{n-3} Q_T.
 *   a9  Ascending eigenvalues; each eigenvector's largest-magnitude entry is
 *       made positive (first index on ties).
 *
 * Pole order follows Eq. (9): within a merge the non-deflated poles are held in
 * DESCENDING order d_1 > d_2 > ... > d_K (0-based: d[0] > d[1] > ...), root i
 * lies in (d_i, d_{i-1}) and root 0 above d_0.
 *
 * Pins: tests/test_oracle_pins.py checks every stage against closed forms,
 * LAPACK, brute-force Jacobi and the paper's identities. Parity unpinned:
 * iteration counts and the section constants k and eps (the paper prints no
 * values); only results are pinned.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U 0x1p-53 /* unit roundoff of IEEE binary64 */
#define ORC_NMAX 256  /* largest n the oracle accepts */

/* Constants the paper leaves unnamed; the caller may override them. */
typedef struct {
    int k_sections;         /* k of Eq. (16) */
    double section_rel_eps; /* Eq. (17): stop when U - L < eps * (initial width) */
    int max_section_iters;  /* cap on multi-section steps */
    int max_halley_iters;   /* cap on Halley steps */
    double stop_c;          /* Halley stops when |f| <= c u (1 + rho sum |z^2/(d-lambda)|) */
    double deflate_c;       /* deflation tolerance = c u max(max|d|, rho |z|^2) */
    int leaf_size;          /* divide until blocks have at most this many rows (1..8); blocks of 3
                               or more rows are solved by the tridiagonal QL iteration */
} orc_opts;

typedef struct {
    int64_t roots;      /* secular roots solved */
    int64_t iters;      /* f evaluations spent on them */
    int64_t deflated;   /* eigenpairs deflated (both kinds) */
    int64_t rotations;  /* close-pole Givens deflations */
    int64_t not_conv;   /* roots that hit an iteration cap */
} orc_stats;

void orc_default_opts(orc_opts* o)
{
    o->k_sections = 4;
    o->section_rel_eps = 0x1p-6;
    o->max_section_iters = 64;
    o->max_halley_iters = 64;
    o->stop_c = 8.0;
    o->deflate_c = 8.0;
    o->leaf_size = 2;
}

static const orc_opts* opts_or_default(const orc_opts* o, orc_opts* tmp)
{
    if (o) return o;
    orc_default_opts(tmp);
    return tmp;
}

/* ------------------------------------------------------------------------ */
/* a1: Householder tridiagonalization                                       */
/* ------------------------------------------------------------------------ */

/*
 * A (n x n, row-major; only the lower triangle is read) = H T H^T with
 * H = H_0 H_1 ... H_{n-3}, H_k = I - tau_k v_k v_k^T, v_k zero above row k+1
 * and v_k[k+1] = 1. T has diagonal d[0..n) and off-diagonal e[0..n-1).
 * Reflector k (LAPACK dlarfg convention): x = A[k+1:, k], alpha = x_0,
 * beta = -sign(alpha) |x|, tau = (beta - alpha)/beta, v = [1, x_1:/(alpha - beta)];
 * H_k x = beta e_1. If x_1: is zero, tau = 0 and beta = alpha.
 * vk (n x n, may be NULL): row k holds v_k. taus (may be NULL): tau_k.
 * H (n x n, may be NULL): the product H_0 ... H_{n-3}.
 */
void orc_tridiagonalize(int n, const double* A, double* d, double* e, double* vk, double* taus,
                        double* H)
{
    double* a = (double*)malloc(sizeof(double) * n * n);
    double* v = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* w = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) a[i * n + j] = (i >= j) ? A[i * n + j] : A[j * n + i];
    if (vk) memset(vk, 0, sizeof(double) * n * n);
    if (H) {
        memset(H, 0, sizeof(double) * n * n);
        for (int i = 0; i < n; i++) H[i * n + i] = 1.0;
    }
    for (int k = 0; k + 2 < n; k++) {
        int m = n - k - 1; /* rows k+1 .. n-1 */
        double alpha = a[(k + 1) * n + k];
        double xn2 = 0;
        for (int i = k + 2; i < n; i++) xn2 += a[i * n + k] * a[i * n + k];
        double tau, beta;
        for (int i = 0; i < n; i++) v[i] = 0;
        v[k + 1] = 1.0;
        if (xn2 == 0.0) {
            tau = 0.0;
            beta = alpha;
        } else {
            double nrm = sqrt(alpha * alpha + xn2);
            beta = (alpha >= 0) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            for (int i = k + 2; i < n; i++) v[i] = a[i * n + k] / (alpha - beta);
        }
        /* two-sided update of the trailing block: a22 <- H_k a22 H_k */
        for (int i = k + 1; i < n; i++) {
            double s = 0;
            for (int j = k + 1; j < n; j++) s += a[i * n + j] * v[j];
            p[i] = tau * s;
        }
        double pv = 0;
        for (int i = k + 1; i < n; i++) pv += p[i] * v[i];
        for (int i = k + 1; i < n; i++) w[i] = p[i] - 0.5 * tau * pv * v[i];
        for (int i = k + 1; i < n; i++)
            for (int j = k + 1; j < n; j++) a[i * n + j] -= v[i] * w[j] + w[i] * v[j];
        /* column k is now beta e_1 below the diagonal */
        for (int i = k + 1; i < n; i++) a[i * n + k] = a[k * n + i] = 0.0;
        a[(k + 1) * n + k] = a[k * n + k + 1] = beta;
        d[k] = a[k * n + k];
        e[k] = beta;
        if (vk)
            for (int i = 0; i < n; i++) vk[k * n + i] = v[i];
        if (taus) taus[k] = tau;
        if (H) { /* H <- H H_k */
            for (int r = 0; r < n; r++) {
                double s = 0;
                for (int j = k + 1; j < n; j++) s += H[r * n + j] * v[j];
                for (int j = k + 1; j < n; j++) H[r * n + j] -= tau * s * v[j];
            }
        }
        (void)m;
    }
    if (n >= 2) {
        d[n - 2] = a[(n - 2) * n + n - 2];
        d[n - 1] = a[(n - 1) * n + n - 1];
        e[n - 2] = a[(n - 1) * n + n - 2];
    } else if (n == 1) {
        d[0] = a[0];
    }
    if (n >= 2 && taus) taus[n - 2] = 0.0;
    free(a);
    free(v);
    free(p);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* a2: tearing, Eq. (2)-(3)                                                 */
/* ------------------------------------------------------------------------ */

/*
 * Tear the s x s tridiagonal (d, e) after row m-1: T = blkdiag(T1^, T2^) + |beta| v v^T
 * with beta = e[m-1], v = [0..0, sign(beta), 1, 0..0] (sign(0) = +1). T1^ and T2^
 * keep their off-diagonals; Eq. (3) subtracts |beta| from the last diagonal entry
 * of T1^ and the first of T2^. d1 gets m entries, d2 gets s - m.
 */
void orc_tear(int s, const double* d, const double* e, int m, double* d1, double* d2, double* rho,
              double* sigma)
{
    double beta = e[m - 1];
    *rho = fabs(beta);
    *sigma = (beta >= 0) ? 1.0 : -1.0;
    for (int i = 0; i < m; i++) d1[i] = d[i];
    for (int i = m; i < s; i++) d2[i - m] = d[i];
    d1[m - 1] -= *rho;
    d2[0] -= *rho;
}

/* ------------------------------------------------------------------------ */
/* a3: 2x2 leaf, Sec. 2.2                                                   */
/* ------------------------------------------------------------------------ */

/*
 * [[a, b], [b, c]] = J diag(a - t b, c + t b) J^T with the Jacobi rotation
 * J = [[cs, sn], [-sn, cs]], t = sn/cs the smaller root of t^2 + 2 theta t - 1 = 0,
 * theta = (c - a)/(2b). Q is row-major; column j is the eigenvector of lam[j].
 */
void orc_eig2(double a, double b, double c, double* lam, double* Q)
{
    if (b == 0.0) {
        lam[0] = a;
        lam[1] = c;
        Q[0] = 1;
        Q[1] = 0;
        Q[2] = 0;
        Q[3] = 1;
        return;
    }
    double theta = (c - a) / (2.0 * b);
    double t = ((theta >= 0) ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    double cs = 1.0 / sqrt(t * t + 1.0);
    double sn = t * cs;
    lam[0] = a - t * b;
    lam[1] = c + t * b;
    Q[0] = cs;
    Q[1] = sn;
    Q[2] = -sn;
    Q[3] = cs;
}

/*
 * a3 (larger leaves): eigendecomposition of the s x s tridiagonal (d, e) by the
 * implicit QL iteration with Wilkinson shifts, following the step recurrence
 * of the EISPACK routine tql2 (Bowdler, Martin, Reinsch and Wilkinson 1968;
 * tqli in Numerical Recipes). For the leading unreduced block
 * [l, mm] (mm the first index with a negligible e[mm]) one step chases the
 * bulge from the bottom: the shift is the eigenvalue of the top 2x2 block of
 * [l, mm] nearer to d[l], and rotations in planes (i, i+1), i = mm-1 .. l,
 * are accumulated into the columns of Q. Output as orc_tridiag_eig: lam
 * ascending, Q row-major with eigenvectors as columns. Returns the number of
 * eigenvalues that hit the iteration cap.
 */
int orc_tridiag_ql(int s, const double* d_in, const double* e_in, double* lam, double* Q)
{
    double d[ORC_NMAX], e[ORC_NMAX];
    int bad = 0;
    for (int i = 0; i < s; i++) {
        d[i] = d_in[i];
        e[i] = (i + 1 < s) ? e_in[i] : 0.0;
        for (int j = 0; j < s; j++) Q[i * s + j] = (i == j) ? 1.0 : 0.0;
    }
    for (int l = 0; l < s; l++) {
        int iter = 0;
        for (;;) {
            int mm = l;
            while (mm < s - 1 && fabs(e[mm]) > ORC_U * (fabs(d[mm]) + fabs(d[mm + 1]))) mm++;
            if (mm == l) break;
            if (++iter > 60) {
                bad++;
                break;
            }
            /* shift: the eigenvalue of [[d_l, e_l], [e_l, d_l+1]] nearer to d_l is d_l - e_l/(g + sign(g) r)
               with g = (d_l+1 - d_l)/(2 e_l), r = sqrt(g^2 + 1); the chase starts from d_mm minus it */
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double sn = 1.0, cs = 1.0, p = 0.0;
            int restarted = 0;
            for (int i = mm - 1; i >= l; i--) {
                double f = sn * e[i], b = cs * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) { /* the bulge vanished: the block splits at i + 1 */
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    restarted = 1;
                    break;
                }
                sn = f / r;
                cs = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * sn + 2.0 * cs * b;
                p = sn * r;
                d[i + 1] = g + p;
                g = cs * r - b;
                for (int k = 0; k < s; k++) { /* columns i, i+1 of Q by the same rotation */
                    double qa = Q[k * s + i], qb = Q[k * s + i + 1];
                    Q[k * s + i + 1] = sn * qa + cs * qb;
                    Q[k * s + i] = cs * qa - sn * qb;
                }
            }
            if (restarted) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    /* ascending order (selection sort, columns of Q follow) */
    for (int i = 0; i < s; i++) {
        int m = i;
        for (int j = i + 1; j < s; j++)
            if (d[j] < d[m]) m = j;
        if (m != i) {
            double t = d[i];
            d[i] = d[m];
            d[m] = t;
            for (int k = 0; k < s; k++) {
                t = Q[k * s + i];
                Q[k * s + i] = Q[k * s + m];
                Q[k * s + m] = t;
            }
        }
    }
    memcpy(lam, d, sizeof(double) * s);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* a5: secular equation                                                     */
/* ------------------------------------------------------------------------ */

/*
 * Eq. (8), (18), (21) at lambda = d[o] + tau: every d_j - lambda is formed as
 * (d_j - d_o) - tau, so that a root next to its pole keeps its relative accuracy.
 * err = 1 + rho sum |z_j^2/(d_j - lambda)| bounds the rounding error of f (in units
 * of u, up to a modest factor).
 */
void orc_secular_eval(int K, const double* d, const double* z, double rho, int o, double tau,
                      double* f, double* f1, double* f2, double* err)
{
    double s0 = 0, s1 = 0, s2 = 0, sa = 0;
    for (int j = 0; j < K; j++) {
        double dl = (d[j] - d[o]) - tau; /* d_j - lambda */
        double t = z[j] * z[j] / dl;
        s0 += t;
        s1 += t / dl;
        s2 += t / (dl * dl);
        sa += fabs(t);
    }
    *f = 1.0 + rho * s0;
    *f1 = rho * s1;
    *f2 = 2.0 * rho * s2;
    *err = 1.0 + rho * sa;
}

/*
 * Root i of f (Eq. (8)) for DESCENDING poles d[0] > ... > d[K-1], z_j != 0, rho > 0.
 * Interlacing Eq. (9)/(11): root i lies in (d_i, d_{i-1}) for i > 0 and in
 * (d_0, upper0] for i = 0. The bracket [L, U] is kept in coordinates relative to
 * a pole d_o. Returns the pole index in *origin and lambda_i - d_origin in *tau.
 */
void orc_secular_root(int K, const double* d, const double* z, double rho, double upper0, int i,
                      const orc_opts* opts, int* origin, double* tau, orc_stats* st)
{
    orc_opts tmp;
    const orc_opts* op = opts_or_default(opts, &tmp);
    double f, f1, f2, err;
    int it = 0, conv = 0;
    if (K == 1) { /* one pole: 1 + rho z^2/(d - lambda) = 0 has lambda = d + rho z^2 */
        *origin = 0;
        *tau = rho * z[0] * z[0];
        if (st) st->roots++;
        return;
    }
    int o = i; /* start relative to the root's lower bound d_i */
    double L = 0.0;
    double U = (i == 0) ? (upper0 - d[0]) : (d[i - 1] - d[i]);
    double width0 = U - L;
    double h;

    /* Eq. (13) (midpoint of the root's own bracket) and one bisection step Eq. (14)-(15) */
    h = 0.5 * (L + U);
    orc_secular_eval(K, d, z, rho, o, h, &f, &f1, &f2, &err);
    it++;
    if (f > 0)
        U = h;
    else if (f < 0)
        L = h;
    else
        conv = 1;
    if (!conv && i > 0 && f < 0) {
        /* root in the upper half: nearer to d_{i-1}; shift the coordinates there */
        double shift = d[i - 1] - d[i];
        o = i - 1;
        L -= shift;
        U = 0.0;
        h -= shift;
    }
    /* multi-section, Eq. (16), until Eq. (17) */
    int ns = 0;
    while (!conv && (U - L) >= op->section_rel_eps * width0 && ns < op->max_section_iters) {
        h = L + (U - L) / op->k_sections;
        orc_secular_eval(K, d, z, rho, o, h, &f, &f1, &f2, &err);
        it++;
        ns++;
        if (f > 0)
            U = h;
        else if (f < 0)
            L = h;
        else
            conv = 1;
    }
    /* Halley's method, Eq. (20)-(21), started at the middle of the bracket */
    if (!conv) {
        h = 0.5 * (L + U);
        int nh = 0;
        for (;;) {
            orc_secular_eval(K, d, z, rho, o, h, &f, &f1, &f2, &err);
            it++;
            if (f == 0.0 || fabs(f) <= op->stop_c * ORC_U * err) {
                conv = 1;
                break;
            }
            if (f > 0)
                U = h;
            else
                L = h;
            if (++nh > op->max_halley_iters) break;
            double den = 2.0 * f1 * f1 - f * f2;
            double hn = h - 2.0 * f * f1 / den;
            /* the top root's upper end is a bound, not a pole, and may be reached */
            int inside = (hn > L) && (i == 0 ? hn <= U : hn < U);
            if (!(den > 0) || !inside) hn = 0.5 * (L + U);
            if (fabs(hn - h) <= 2.0 * ORC_U * fabs(hn)) {
                h = hn;
                conv = 1;
                break;
            }
            h = hn;
        }
    }
    *origin = o;
    *tau = h;
    if (st) {
        st->roots++;
        st->iters += it;
        if (!conv) st->not_conv++;
    }
}

/*
 * Eq. (25): z-hat_i = sqrt( prod_j (lambda_j - d_i) / (rho prod_{j != i} (d_j - d_i)) ),
 * given the roots as (origin, tau) pairs over the same DESCENDING poles; the sign is taken
 * from z_i. lambda_j - d_i is formed as (d_{o_j} - d_i) + tau_j.
 * The two products of Eq. (25) under- or overflow once many poles cluster (K factors of size
 * 1e-9 already underflow binary64), so the same quotient is evaluated as the product of
 * interlaced ratios, each in (0, 1) by Eq. (9):
 *   (lambda_0 - d_i)/rho * prod_{j<i} (lambda_{j+1} - d_i)/(d_j - d_i)
 *                        * prod_{j>i} (lambda_j - d_i)/(d_j - d_i),
 * starting with the one factor that may exceed 1, so no partial product leaves the range
 * of the result.
 */
void orc_loewner_zhat(int K, const double* d, const double* z, double rho, const int* origin,
                      const double* tau, double* zhat)
{
    for (int i = 0; i < K; i++) {
        double q = ((d[origin[0]] - d[i]) + tau[0]) / rho;
        for (int j = 0; j < i; j++) q *= ((d[origin[j + 1]] - d[i]) + tau[j + 1]) / (d[j] - d[i]);
        for (int j = i + 1; j < K; j++) q *= ((d[origin[j]] - d[i]) + tau[j]) / (d[j] - d[i]);
        zhat[i] = (z[i] >= 0 ? 1.0 : -1.0) * sqrt(q > 0 ? q : 0.0);
    }
}

/* ------------------------------------------------------------------------ */
/* a4-a6: eigendecomposition of D + rho z z^T                               */
/* ------------------------------------------------------------------------ */

static void sort_pairs_ascending(int s, double* lam, double* Q /* s x s, columns */)
{
    /* plain selection sort of eigenpairs (stable by index on ties) */
    double* col = (double*)malloc(sizeof(double) * s);
    for (int a = 0; a < s; a++) {
        int m = a;
        for (int b = a + 1; b < s; b++)
            if (lam[b] < lam[m]) m = b;
        if (m != a) {
            /* rotate entries a..m right by one to keep equal keys in index order */
            double lm = lam[m];
            for (int r = 0; r < s; r++) col[r] = Q[r * s + m];
            for (int b = m; b > a; b--) {
                lam[b] = lam[b - 1];
                for (int r = 0; r < s; r++) Q[r * s + b] = Q[r * s + b - 1];
            }
            lam[a] = lm;
            for (int r = 0; r < s; r++) Q[r * s + a] = col[r];
        }
    }
    free(col);
}

/*
 * Eigendecomposition of D + rho z z^T (the middle factor of Eq. (4)), rho >= 0.
 * D[s] and z[s] are in the children's column order. lam[s] comes out ascending
 * and Uq (s x s, row-major) holds the eigenvectors as columns.
 *
 * Deflation (reading; the paper does not describe it): with
 * tol = deflate_c u max(max|d|, rho |z|^2),
 *   (i)  rho |z_i| |z| <= tol          -> (d_i, e_i) is an eigenpair;
 *   (ii) for consecutive surviving poles (in the order of Eq. (9)), with
 *        r = hypot(z_a, z_b), c = z_b/r, s = z_a/r: if |(d_b - d_a) c s| <= tol,
 *        a Givens rotation moves all of the coupling to b and a is deflated.
 */
void orc_rank_one_eig(int s, const double* D, const double* z, double rho, const orc_opts* opts,
                      double* lam, double* Uq, orc_stats* st)
{
    orc_opts tmp;
    const orc_opts* op = opts_or_default(opts, &tmp);
    int* perm = (int*)malloc(sizeof(int) * s);
    int* defl = (int*)malloc(sizeof(int) * s);
    int* rot_j = (int*)malloc(sizeof(int) * s);
    int* idx = (int*)malloc(sizeof(int) * s);
    int* orig = (int*)malloc(sizeof(int) * s);
    double* dd = (double*)malloc(sizeof(double) * s);
    double* zz = (double*)malloc(sizeof(double) * s);
    double* rc = (double*)malloc(sizeof(double) * s);
    double* rs = (double*)malloc(sizeof(double) * s);
    double* dK = (double*)malloc(sizeof(double) * s);
    double* zK = (double*)malloc(sizeof(double) * s);
    double* tau = (double*)malloc(sizeof(double) * s);
    double* zh = (double*)malloc(sizeof(double) * s);
    double* Y = (double*)calloc((size_t)s * s, sizeof(double));
    double* mu = (double*)malloc(sizeof(double) * s);

    /* order the poles as in Eq. (9): descending, ties by index */
    for (int p = 0; p < s; p++) perm[p] = p;
    for (int a = 1; a < s; a++) { /* insertion sort, stable */
        int x = perm[a], b = a - 1;
        while (b >= 0 && D[perm[b]] < D[x]) {
            perm[b + 1] = perm[b];
            b--;
        }
        perm[b + 1] = x;
    }
    double nz2 = 0, dmax = 0;
    for (int p = 0; p < s; p++) {
        dd[p] = D[perm[p]];
        zz[p] = z[perm[p]];
        nz2 += zz[p] * zz[p];
        if (fabs(dd[p]) > dmax) dmax = fabs(dd[p]);
        rot_j[p] = -1;
    }
    double nz = sqrt(nz2);
    double tol = op->deflate_c * ORC_U * fmax(dmax, rho * nz2);

    /* deflation (i) */
    for (int p = 0; p < s; p++) defl[p] = (rho * fabs(zz[p]) * nz <= tol);
    /* deflation (ii), one pass in pole order */
    int pj = -1;
    for (int p = 0; p < s; p++) {
        if (defl[p]) continue;
        if (pj < 0) {
            pj = p;
            continue;
        }
        double r = hypot(zz[pj], zz[p]);
        double c = zz[p] / r, sn = zz[pj] / r;
        if (fabs((dd[p] - dd[pj]) * c * sn) <= tol) {
            double a = dd[pj], b = dd[p];
            dd[pj] = c * c * a + sn * sn * b;
            dd[p] = sn * sn * a + c * c * b;
            zz[p] = r;
            zz[pj] = 0.0;
            defl[pj] = 1;
            rot_j[pj] = p;
            rc[pj] = c;
            rs[pj] = sn;
            if (st) st->rotations++;
        }
        pj = p;
    }
    int K = 0;
    for (int p = 0; p < s; p++)
        if (!defl[p]) {
            idx[K] = p;
            dK[K] = dd[p];
            zK[K] = zz[p];
            K++;
        }
    if (st) st->deflated += s - K;

    /* a5: roots, Eq. (8)-(21) */
    if (K > 0) {
        double zn2 = 0, fro2 = 0, dz = 0;
        for (int i = 0; i < K; i++) {
            zn2 += zK[i] * zK[i];
            fro2 += dK[i] * dK[i];
            dz += dK[i] * zK[i] * zK[i];
        }
        /* Eq. (10)-(11): lambda_0 <= |D + rho z z^T|_F, and lambda_0 <= d_0 + rho |z|^2 */
        fro2 += 2.0 * rho * dz + rho * rho * zn2 * zn2;
        double up = dK[0] + rho * zn2;
        double fro = sqrt(fro2);
        if (fro < up && fro > dK[0]) up = fro;
        for (int i = 0; i < K; i++) orc_secular_root(K, dK, zK, rho, up, i, op, &orig[i], &tau[i], st);
        /* a6: Eq. (25) then Eq. (24) */
        orc_loewner_zhat(K, dK, zK, rho, orig, tau, zh);
    }
    int col = 0;
    for (int j = 0; j < K; j++, col++) {
        double nrm = 0;
        for (int i = 0; i < K; i++) {
            double q = zh[i] / ((dK[i] - dK[orig[j]]) - tau[j]); /* z^_i / (d_i - lambda_j) */
            Y[idx[i] * s + col] = q;
            nrm += q * q;
        }
        nrm = sqrt(nrm);
        for (int i = 0; i < K; i++) Y[idx[i] * s + col] /= nrm;
        mu[col] = dK[orig[j]] + tau[j];
    }
    for (int p = 0; p < s; p++)
        if (defl[p]) {
            Y[p * s + col] = 1.0;
            mu[col] = dd[p];
            col++;
        }
    /* undo the Givens rotations, last one first: x = G_1 (G_2 (... y)) */
    for (int p = s - 1; p >= 0; p--) {
        if (rot_j[p] < 0) continue;
        int q = rot_j[p];
        double c = rc[p], sn = rs[p];
        for (int k = 0; k < s; k++) {
            double yp = Y[p * s + k], yq = Y[q * s + k];
            Y[p * s + k] = c * yp + sn * yq;
            Y[q * s + k] = -sn * yp + c * yq;
        }
    }
    /* undo the pole ordering */
    for (int p = 0; p < s; p++)
        for (int k = 0; k < s; k++) Uq[perm[p] * s + k] = Y[p * s + k];
    for (int k = 0; k < s; k++) lam[k] = mu[k];
    sort_pairs_ascending(s, lam, Uq);

    free(perm);
    free(defl);
    free(rot_j);
    free(idx);
    free(orig);
    free(dd);
    free(zz);
    free(rc);
    free(rs);
    free(dK);
    free(zK);
    free(tau);
    free(zh);
    free(Y);
    free(mu);
}

/* ------------------------------------------------------------------------ */
/* a2-a7: divide and conquer on the tridiagonal                             */
/* ------------------------------------------------------------------------ */

/*
 * Eigendecomposition of the s x s tridiagonal (d, e): T = Q diag(lam) Q^T,
 * lam ascending, Q row-major with eigenvectors as columns. Sec. 2.1: tear at
 * m = floor(s/2) (Eq. (2)-(3)), solve both halves recursively down to blocks of
 * at most leaf_size rows (Sec. 2.2), then merge through Eq. (4)-(5).
 */
void orc_tridiag_eig(int s, const double* d, const double* e, const orc_opts* opts, double* lam,
                     double* Q, orc_stats* st)
{
    orc_opts tmp;
    const orc_opts* op = opts_or_default(opts, &tmp);
    if (s == 1) {
        lam[0] = d[0];
        Q[0] = 1.0;
        return;
    }
    if (s >= 3 && s <= op->leaf_size) {
        int bad = orc_tridiag_ql(s, d, e, lam, Q);
        if (st) st->not_conv += bad;
        return;
    }
    if (s == 2 && op->leaf_size >= 2) {
        double l2[2], q2[4];
        orc_eig2(d[0], e[0], d[1], l2, q2);
        /* ascending order */
        if (l2[1] < l2[0]) {
            lam[0] = l2[1];
            lam[1] = l2[0];
            Q[0] = q2[1];
            Q[1] = q2[0];
            Q[2] = q2[3];
            Q[3] = q2[2];
        } else {
            memcpy(lam, l2, sizeof l2);
            memcpy(Q, q2, sizeof q2);
        }
        return;
    }
    int m = s / 2, s2 = s - m;
    double rho, sigma;
    double* d1 = (double*)malloc(sizeof(double) * m);
    double* d2 = (double*)malloc(sizeof(double) * s2);
    double* l1 = (double*)malloc(sizeof(double) * m);
    double* l2 = (double*)malloc(sizeof(double) * s2);
    double* Q1 = (double*)malloc(sizeof(double) * m * m);
    double* Q2 = (double*)malloc(sizeof(double) * s2 * s2);
    double* D = (double*)malloc(sizeof(double) * s);
    double* z = (double*)malloc(sizeof(double) * s);
    double* Uq = (double*)malloc(sizeof(double) * s * s);
    orc_tear(s, d, e, m, d1, d2, &rho, &sigma);
    orc_tridiag_eig(m, d1, e, op, l1, Q1, st);
    orc_tridiag_eig(s2, d2, e + m, op, l2, Q2, st);
    /* Eq. (4)-(5): D = diag(D1, D2); z = blkdiag(Q1, Q2)^T v
       = [sigma * (last row of Q1)^T ; (first row of Q2)^T] */
    for (int j = 0; j < m; j++) {
        D[j] = l1[j];
        z[j] = sigma * Q1[(m - 1) * m + j];
    }
    for (int j = 0; j < s2; j++) {
        D[m + j] = l2[j];
        z[m + j] = Q2[j];
    }
    orc_rank_one_eig(s, D, z, rho, op, lam, Uq, st);
    /* a7: Q = blkdiag(Q1, Q2) Uq */
    for (int r = 0; r < s; r++)
        for (int c = 0; c < s; c++) {
            double acc = 0;
            if (r < m)
                for (int k = 0; k < m; k++) acc += Q1[r * m + k] * Uq[k * s + c];
            else
                for (int k = 0; k < s2; k++) acc += Q2[(r - m) * s2 + k] * Uq[(m + k) * s + c];
            Q[r * s + c] = acc;
        }
    free(d1);
    free(d2);
    free(l1);
    free(l2);
    free(Q1);
    free(Q2);
    free(D);
    free(z);
    free(Uq);
}

/* ------------------------------------------------------------------------ */
/* a1-a9: the whole path for one matrix                                     */
/* ------------------------------------------------------------------------ */

/*
 * A (n x n, row-major, lower triangle read) = V diag(W) V^T; W ascending,
 * V row-major with eigenvector j in column j, its largest-|.| entry positive.
 */
void orc_eigh(int n, const double* A, const orc_opts* opts, double* W, double* V, orc_stats* st)
{
    orc_opts tmp;
    const orc_opts* op = opts_or_default(opts, &tmp);
    if (n <= 0) return;
    double* d = (double*)malloc(sizeof(double) * n);
    double* e = (double*)malloc(sizeof(double) * n);
    double* H = (double*)malloc(sizeof(double) * n * n);
    double* QT = (double*)malloc(sizeof(double) * n * n);
    orc_tridiagonalize(n, A, d, e, NULL, NULL, H);
    orc_tridiag_eig(n, d, e, op, W, QT, st);
    /* a8: V = H Q_T */
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            double acc = 0;
            for (int k = 0; k < n; k++) acc += H[r * n + k] * QT[k * n + c];
            V[r * n + c] = acc;
        }
    /* a9: W is ascending already; sign of each column */
    for (int c = 0; c < n; c++) {
        int im = 0;
        for (int r = 1; r < n; r++)
            if (fabs(V[r * n + c]) > fabs(V[im * n + c])) im = r;
        if (V[im * n + c] < 0)
            for (int r = 0; r < n; r++) V[r * n + c] = -V[r * n + c];
    }
    free(d);
    free(e);
    free(H);
    free(QT);
}

/* ------------------------------------------------------------------------ */
/* gradient of a loss of (W, V) with respect to A                          */
/* ------------------------------------------------------------------------ */

/*
 * Reverse-mode derivative of the eigendecomposition A = V diag(W) V^T (the eigendecomposition layer the
 * paper's introduction motivates): with first-order perturbation theory,
 * dW_i = v_i^T dA v_i and dv_i = sum_{j != i} v_j (v_j^T dA v_i)/(W_i - W_j), so for gW = dL/dW and
 * gV = dL/dV,
 *     G = V (diag(gW) + F o (V^T gV)) V^T,   F_ij = 1/(W_j - W_i) for i != j, F_ii = 0,
 * and gA = (G + G^T)/2, the gradient over symmetric perturbations of A. Pairs with
 * |W_j - W_i| <= gap_eps get F_ij = 0 (their eigenvectors are not determined individually).
 * gW or gV may be NULL (zero). All n x n arrays row-major, V with eigenvectors in columns.
 */
void orc_eigh_backward(int n, const double* W, const double* V, const double* gW, const double* gV,
                       double gap_eps, double* gA)
{
    double* M = (double*)calloc((size_t)n * n, sizeof(double));
    double* T = (double*)calloc((size_t)n * n, sizeof(double));
    double* G = (double*)calloc((size_t)n * n, sizeof(double));
    /* M = diag(gW) + F o (V^T gV) */
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double m = 0;
            if (i == j) {
                m = gW ? gW[i] : 0.0;
            } else if (gV && fabs(W[j] - W[i]) > gap_eps) {
                double vg = 0;
                for (int k = 0; k < n; k++) vg += V[k * n + i] * gV[k * n + j];
                m = vg / (W[j] - W[i]);
            }
            M[i * n + j] = m;
        }
    /* G = V M V^T */
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0;
            for (int k = 0; k < n; k++) acc += V[i * n + k] * M[k * n + j];
            T[i * n + j] = acc;
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0;
            for (int k = 0; k < n; k++) acc += T[i * n + k] * V[j * n + k];
            G[i * n + j] = acc;
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) gA[i * n + j] = 0.5 * (G[i * n + j] + G[j * n + i]);
    free(M);
    free(T);
    free(G);
}

/* ------------------------------------------------------------------------ */
/* batch driver (plain threads over independent matrices)                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t lo, hi;
    int n;
    const float* A;
    double* W;
    double* V;
    const orc_opts* op;
    orc_stats st;
} orc_job;

static void* orc_worker(void* arg)
{
    orc_job* j = (orc_job*)arg;
    int n = j->n;
    double* a = (double*)malloc(sizeof(double) * n * n);
    for (int64_t b = j->lo; b < j->hi; b++) {
        for (int i = 0; i < n * n; i++) a[i] = (double)j->A[b * n * n + i];
        orc_eigh(n, a, j->op, j->W + b * n, j->V + b * n * n, &j->st);
    }
    free(a);
    return NULL;
}

/*
 * Batched entry: A is batch x n x n FP32 (upcast exactly to FP64), W batch x n,
 * V batch x n x n (FP64). nthreads <= 1 runs on the calling thread. Returns the
 * number of threads used. st (may be NULL) receives the summed counters.
 */
int orc_eigh_batch_f32(int64_t batch, int n, const float* A, const orc_opts* opts, double* W,
                       double* V, int nthreads, orc_stats* st)
{
    orc_opts tmp;
    const orc_opts* op = opts_or_default(opts, &tmp);
    if (n <= 0 || n > ORC_NMAX || batch <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > batch) nthreads = (int)batch;
    orc_job* jobs = (orc_job*)calloc(nthreads, sizeof(orc_job));
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        jobs[t].lo = batch * t / nthreads;
        jobs[t].hi = batch * (t + 1) / nthreads;
        jobs[t].n = n;
        jobs[t].A = A;
        jobs[t].W = W;
        jobs[t].V = V;
        jobs[t].op = op;
    }
    if (nthreads == 1)
        orc_worker(&jobs[0]);
    else {
        for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    }
    if (st) {
        memset(st, 0, sizeof *st);
        for (int t = 0; t < nthreads; t++) {
            st->roots += jobs[t].st.roots;
            st->iters += jobs[t].st.iters;
            st->deflated += jobs[t].st.deflated;
            st->rotations += jobs[t].st.rotations;
            st->not_conv += jobs[t].st.not_conv;
        }
    }
    free(jobs);
    free(th);
    return nthreads;
}
