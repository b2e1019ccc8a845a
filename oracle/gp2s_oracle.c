/*
 * gp2s_oracle.c -- plain FP64 CPU oracle for the exact sparse-kernel Gaussian-process
 * log marginal likelihood of gp2Scale (Noack, Risser, Luo, Tekriwal, Pandolfi,
 * arXiv 2512.06143).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check (__graft_entry__.smoke) and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source, header, table
 * or helper with the CUDA path under paper_2512_06143_gb300/, and it never calls it.
 *
 * Everything here is the plain definition, written out in FP64, one pair / one row at a
 * time, in the order the paper states it:
 *   - Eq. 3, Sec. 4.1: the compactly supported Wendland taper, strict support t < 1;
 *   - Eq. 7, Sec. 4.3: bump functions b(x) = a exp(beta (1 - 1/(1 - s))), s = |x-c|^2/rho^2;
 *   - the product kernel of Sec. 4.1 with a rank-<=L bump factor (Sec. 4.3, Theorem 1):
 *       k(xi, xj) = phi(|xi - xj| / r) * (sum_l b_l(xi) b_l(xj) + w0);
 *   - Sec. 3 (Background): A = K + sigma^2 I, the LML needs a = A^{-1} y and log|A|;
 *   - Sec. 4.6: the paper evaluates every covariance entry -> brute-force all-pairs assembly.
 * Krylov pieces (conjugate gradients, Lanczos) follow their textbook definitions; they are
 * used only where the paper leaves the log-determinant method open (Sec. 4.6, App. B.7).
 *
 * Readings taken where the paper is silent or garbled:
 *   - "Wendland C2" = phi(t) = (1-t)^4 (4t+1) for d <= 3 and (1-t)^5 (5t+1) for d = 4;
 *     Eq. 3's own C6 form (1-t)^8 (32t^3+25t^2+8t+1) is kind 1.
 *   - bump support is s = |x-c|^2 / rho^2 < 1 (Eq. 7 prints "|x-c|^2 < r").
 *   - the pattern is structural: (i, j) is stored iff i == j or d2(i, j) < r*r, where
 *     d2 = ((D0*D0 + D1*D1) + D2*D2) + ...,  Dk = xi[k] - xj[k], every operation one FP64
 *     round-to-nearest step and no fused multiply-add (build with -ffp-contract=off).
 *   - probes are Rademacher signs from SplitMix64 (Vigna), indexed by the original point index.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Hyperparameters of the kernel (Sec. 4.1 + Sec. 4.3) and the noise (Sec. 3). */
typedef struct {
    int d;                 /* input dimension, 1..4 */
    int L;                 /* number of bumps (U = L groups with P = 1 bump each, Sec. 4.3) */
    int kind;              /* 0 = Wendland C2 (reading), 1 = Eq. 3 C6 */
    int pad_;
    double r;              /* Wendland support radius r0 */
    double sigma2;         /* noise variance: V = sigma2 * I */
    double beta;           /* bump shape parameter */
    double w0;             /* constant added to the bump sum (stationary floor, Sec. 4.3) */
    const double *centers; /* L x d, row-major */
    const double *radii;   /* L */
    const double *amps;    /* L */
    int family;            /* 0 = product kernel (Sec. 4.1 / 4.3), 1 = Wendland convolution (Eq. 6) */
    int pad2_;
    const double *ell;     /* family 1: d base length-scale factors */
    const double *G;       /* family 1: L x d weights of the length-scale field */
} orc_hyper;

/* ------------------------------------------------------------------------------------ */
/* SplitMix64 (S. Vigna, public-domain reference generator): the first output of a      */
/* generator whose 64-bit state starts at x.                                            */
/* ------------------------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Rademacher probe s (1-based; s = 0 is reserved) at original point index i:
 * z = +1 if the top bit of splitmix64(seed XOR (s * 2^32 + i)) is 0, else -1.
 * Output layout: z[i * m + (s - 1)], i.e. an n x m row-major matrix. */
void orc_rademacher(int64_t n, int m, uint64_t seed, double *z)
{
    for (int64_t i = 0; i < n; ++i)
        for (int s = 1; s <= m; ++s) {
            uint64_t key = seed ^ (((uint64_t)s << 32) + (uint64_t)i);
            uint64_t bit = orc_splitmix64(key) >> 63;
            z[i * m + (s - 1)] = 1.0 - 2.0 * (double)bit;
        }
}

/* ------------------------------------------------------------------------------------ */
/* Wendland taper phi(t), t = |xi - xj| / r (Eq. 3), and d phi / d t.          */
/* ------------------------------------------------------------------------------------ */
double orc_phi(int kind, int d, double t)
{
    if (!(t < 1.0)) return 0.0;          /* compact support: zero for t >= 1 */
    if (t < 0.0) t = 0.0;
    double u = 1.0 - t;
    if (kind == 1) {                     /* Eq. 3: (1-t)^8 (32 t^3 + 25 t^2 + 8 t + 1) */
        double u2 = u * u, u4 = u2 * u2, u8 = u4 * u4;
        return u8 * (32.0 * t * t * t + 25.0 * t * t + 8.0 * t + 1.0);
    }
    if (d <= 3) {                        /* C2 reading, valid up to R^3: (1-t)^4 (4t+1) */
        double u2 = u * u;
        return u2 * u2 * (4.0 * t + 1.0);
    }
    {                                    /* C2 reading for R^4: (1-t)^5 (5t+1) */
        double u2 = u * u;
        return u2 * u2 * u * (5.0 * t + 1.0);
    }
}

double orc_dphi(int kind, int d, double t)
{
    if (!(t < 1.0)) return 0.0;
    if (t < 0.0) t = 0.0;
    double u = 1.0 - t;
    if (kind == 1) {                     /* derivative of Eq. 3 */
        double u2 = u * u, u4 = u2 * u2, u7 = u4 * u2 * u;
        return -22.0 * t * u7 * (16.0 * t * t + 7.0 * t + 1.0);
    }
    if (d <= 3) return -20.0 * t * u * u * u;
    return -30.0 * t * u * u * u * u;
}

/* phi'(t) / t, finite at t = 0 (the derivative of each form carries a factor t). */
double orc_dphi_over_t(int kind, int d, double t)
{
    if (!(t < 1.0)) return 0.0;
    if (t < 0.0) t = 0.0;
    double u = 1.0 - t;
    if (kind == 1) {
        double u2 = u * u, u4 = u2 * u2, u7 = u4 * u2 * u;
        return -22.0 * u7 * (16.0 * t * t + 7.0 * t + 1.0);
    }
    if (d <= 3) return -20.0 * u * u * u;
    return -30.0 * u * u * u * u;
}

/* ------------------------------------------------------------------------------------ */
/* Bump functions of Eq. 7: b_l(x) = a_l exp(beta (1 - 1/(1 - s))), s = |x-c_l|^2/rho_l^2,
 * zero for s >= 1.  Optionally the derivatives with respect to the bump's parameters,
 * db[l*(d+2) + k] = d b_l / d c_{l,k} (k < d), db[l*(d+2)+d] = d b_l / d rho_l,
 * db[l*(d+2)+d+1] = d b_l / d a_l.                                                     */
/* ------------------------------------------------------------------------------------ */
void orc_bumps(const orc_hyper *h, const double *x, double *b, double *db)
{
    const int d = h->d;
    for (int l = 0; l < h->L; ++l) {
        const double *c = h->centers + (size_t)l * d;
        double rho = h->radii[l], a = h->amps[l];
        double q = 0.0;
        for (int k = 0; k < d; ++k) {
            double dk = x[k] - c[k];
            q = q + dk * dk;
        }
        double s = q / (rho * rho);
        double e = 0.0;                  /* b / a */
        if (s < 1.0) e = exp(h->beta * (1.0 - 1.0 / (1.0 - s)));
        b[l] = a * e;
        if (db) {
            double *g = db + (size_t)l * (d + 2);
            if (s < 1.0 && e > 0.0) {
                double om = 1.0 - s;
                double bl = a * e;
                /* d b / d s = -beta b / (1 - s)^2 */
                double dbds = -h->beta * bl / (om * om);
                for (int k = 0; k < d; ++k)       /* d s / d c_k = -2 (x_k - c_k) / rho^2 */
                    g[k] = dbds * (-2.0 * (x[k] - c[k]) / (rho * rho));
                g[d] = dbds * (-2.0 * s / rho);   /* d s / d rho = -2 s / rho */
                g[d + 1] = e;                     /* d b / d a */
            } else {
                for (int k = 0; k < d + 2; ++k) g[k] = 0.0;
            }
        }
    }
}

/* Squared distance in the pattern's fixed FP64 order (no fused multiply-add). */
double orc_sqdist(int d, const double *xi, const double *xj)
{
    double q = 0.0;
    for (int k = 0; k < d; ++k) {
        double dk = xi[k] - xj[k];
        double sq = dk * dk;
        q = q + sq;
    }
    return q;
}

/* Structural pattern test: stored iff i == j or d2 < r*r (strict, Eq. 3). */
int orc_in_pattern(int d, const double *xi, const double *xj, double r)
{
    double r2 = r * r;
    return orc_sqdist(d, xi, xj) < r2;
}

/* Kernel value k(xi, xj) (no noise term) from precomputed bump values bi, bj. */
static double kernel_from_bumps(const orc_hyper *h, const double *xi, const double *xj,
                                const double *bi, const double *bj)
{
    double q = orc_sqdist(h->d, xi, xj);
    double t = sqrt(q) / h->r;
    double s = 0.0;
    for (int l = 0; l < h->L; ++l) s = s + bi[l] * bj[l];
    return orc_phi(h->kind, h->d, t) * (s + h->w0);
}



/* ------------------------------------------------------------------------------------ */
/* Wendland convolution kernel (Eq. 6, Sec. 4.2), family 1:                              */
/*   k(xi, xj) = s(xi) s(xj) |S_i|^(1/4) |S_j|^(1/4) / |(S_i + S_j)/2|^(1/2) phi(sqrt(Q)/r0), */
/*   Q = (xi - xj)^T ((S_i + S_j)/2)^{-1} (xi - xj),  support Q < r0^2.                    */
/* The paper leaves the fields s (signal deviation) and S (length scale) parametric.      */
/* Reading: S(x) = diag(lambda_1(x), .., lambda_d(x)) with                               */
/*   lambda_k(x) = ell_k^2 + sum_l G_lk psi_l(x),   s(x) = w0 + sum_l a_l psi_l(x),       */
/*   psi_l(x) = (1 - q_l / rho_l^2)^3 for q_l = |x - c_l|^2 < rho_l^2, else 0,            */
/* a polynomial bump on the bumps' centers and radii.  With G = 0, ell = 1, a = 0, w0 = 1 */
/* the kernel is Eq. 3's stationary Wendland taper.  Every step of lambda and Q is one    */
/* FP64 round-to-nearest operation in the order written (the pattern depends on it).     */
/* ------------------------------------------------------------------------------------ */
static double wc_psi(const orc_hyper *h, int l, const double *x, double *s_out)
{
    const int d = h->d;
    const double *c = h->centers + (size_t)l * d;
    double q = 0.0;
    for (int k = 0; k < d; ++k) {
        double dk = x[k] - c[k];
        q = q + dk * dk;
    }
    double rho = h->radii[l];
    double s = q / (rho * rho);
    if (s_out) *s_out = s;
    if (!(s < 1.0)) return 0.0;
    double u = 1.0 - s;
    return u * u * u;
}

/* [s(x), lambda_0(x), .., lambda_{d-1}(x)] */
static void wc_point(const orc_hyper *h, const double *x, double *out)
{
    const int d = h->d, L = h->L;
    double sig = 0.0, acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < L; ++l) {
        double psi = wc_psi(h, l, x, NULL);
        sig = sig + h->amps[l] * psi;
        for (int k = 0; k < d; ++k) acc[k] = acc[k] + h->G[(size_t)l * d + k] * psi;
    }
    out[0] = h->w0 + sig;
    for (int k = 0; k < d; ++k) out[1 + k] = h->ell[k] * h->ell[k] + acc[k];
}

/* Q(i, j) = ((D0 D0 / m0 + D1 D1 / m1) + ...), m_k = (lambda_ik + lambda_jk) * 0.5 */
double orc_wc_q(int d, const double *xi, const double *xj, const double *li, const double *lj)
{
    double q = 0.0;
    for (int k = 0; k < d; ++k) {
        double dk = xi[k] - xj[k];
        double m = (li[k] + lj[k]) * 0.5;
        q = q + (dk * dk) / m;
    }
    return q;
}

/* ------------------------------------------------------------------------------------ */
/* Far-field kernel (Sec. 4.5, the extension for small core length scales), family 2:    */
/*   k(xi, xj) = w0 phi(|xi - xj| / r) + kappa(|xi - xj|) sum_l b_l(xi) b_l(xj),          */
/*   kappa(rho) = exp(-rho^2 / (2 lc^2)),                                                */
/* a local Wendland term (k_core1 = w0, constant) plus the bumps' far-field term tied to a */
/* globally supported squared-exponential core k_core2 = kappa (lc = ell[0]), active only  */
/* inside the bumps' support.  Pattern: i == j, or d2 < r^2, or both points strictly inside */
/* one bump (s_l < 1, s_l = q_l / (rho_l rho_l) in the FP64 order of Eq. 7's bumps).       */
/* ------------------------------------------------------------------------------------ */
static void ff_point(const orc_hyper *h, const double *x, double *out)
{
    const int L = h->L, d = h->d;
    orc_bumps(h, x, out, NULL);
    for (int l = 0; l < L; ++l) {
        const double *c = h->centers + (size_t)l * d;
        double q = 0.0;
        for (int k = 0; k < d; ++k) {
            double dk = x[k] - c[k];
            q = q + dk * dk;
        }
        double rho = h->radii[l];
        out[L + l] = (q / (rho * rho)) < 1.0 ? 1.0 : 0.0;
    }
}

static double ff_kappa(const orc_hyper *h, double q) { return exp(-q / (2.0 * h->ell[0] * h->ell[0])); }

static int point_width(const orc_hyper *h)
{
    if (h->family == 1) return h->d + 1;
    if (h->family == 2) return 2 * h->L;
    return h->L;
}

static void point_values(const orc_hyper *h, const double *x, double *out)
{
    if (h->family == 1) wc_point(h, x, out);
    else if (h->family == 2) ff_point(h, x, out);
    else orc_bumps(h, x, out, NULL);
}

/* Pattern test of two distinct points (the diagonal is always stored). */
static int pair_in(const orc_hyper *h, const double *xi, const double *xj, const double *pi, const double *pj)
{
    if (h->family == 1) return orc_wc_q(h->d, xi, xj, pi + 1, pj + 1) < h->r * h->r;
    if (h->family == 2) {
        if (orc_in_pattern(h->d, xi, xj, h->r)) return 1;
        for (int l = 0; l < h->L; ++l)
            if (pi[h->L + l] != 0.0 && pj[h->L + l] != 0.0) return 1;
        return 0;
    }
    return orc_in_pattern(h->d, xi, xj, h->r);
}

/* Kernel value k(xi, xj) (no noise term) from the points' values. */
static double pair_value(const orc_hyper *h, const double *xi, const double *xj, const double *pi, const double *pj)
{
    if (h->family == 2) {
        double q = orc_sqdist(h->d, xi, xj);
        double loc = q < h->r * h->r ? h->w0 * orc_phi(h->kind, h->d, sqrt(q) / h->r) : 0.0;
        double sb = 0.0;
        for (int l = 0; l < h->L; ++l) sb = sb + pi[l] * pj[l];
        return loc + ff_kappa(h, q) * sb;
    }
    if (h->family != 1) return kernel_from_bumps(h, xi, xj, pi, pj);
    const int d = h->d;
    double q = orc_wc_q(d, xi, xj, pi + 1, pj + 1);
    double pref = 1.0;
    for (int k = 0; k < d; ++k) {
        double li = pi[1 + k], lj = pj[1 + k];
        pref = pref * sqrt(sqrt(li * lj)) / sqrt((li + lj) * 0.5);
    }
    return pi[0] * pj[0] * pref * orc_phi(h->kind, d, sqrt(q) / h->r);
}

double orc_kernel(const orc_hyper *h, const double *xi, const double *xj)
{
    double bi[64], bj[64];
    if (point_width(h) > 64) return NAN;
    point_values(h, xi, bi);
    point_values(h, xj, bj);
    return pair_value(h, xi, xj, bi, bj);
}

/* Per-point values for n points (n x point_width), for the pins and for choosing the
 * k-d tree radius of the candidate search. */
void orc_point_values(const orc_hyper *h, int64_t n, const double *X, double *out)
{
    const int w = point_width(h);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) point_values(h, X + (size_t)i * h->d, out + (size_t)i * w);
}

/* Point table (n x point_width): the bump values b_l(x_i) (family 0) or [s, lambda] (family
 * 1) of every point (the definition evaluated once per point). */
static double *bump_table(int64_t n, const double *X, const orc_hyper *h)
{
    const int w = point_width(h);
    double *B = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(w > 0 ? w : 1));
    if (!B) return NULL;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) point_values(h, X + (size_t)i * h->d, B + (size_t)i * w);
    return B;
}

/* ------------------------------------------------------------------------------------ */
/* Brute-force all-pairs assembly of A = K + sigma^2 I in CSR, original index order,    */
/* columns ascending (Sec. 4.6: every pair is evaluated).                               */
/*   rowptr: n+1 int64 (always written).  col/val: written when non-NULL (pass NULL on  */
/*   a first call to learn nnz = rowptr[n]).  Returns nnz, or -1 on allocation failure. */
/* ------------------------------------------------------------------------------------ */
int64_t orc_assemble_brute(int64_t n, const double *X, const orc_hyper *h,
                           int64_t *rowptr, int32_t *col, double *val)
{
    const int d = h->d, w = point_width(h);
    double *B = bump_table(n, X, h);
    if (!B) return -1;
    if (!col) {
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = 0;
            for (int64_t j = 0; j < n; ++j)
                if (j == i || pair_in(h, X + (size_t)i * d, X + (size_t)j * d, B + (size_t)i * w, B + (size_t)j * w)) ++c;
            rowptr[i + 1] = c;
        }
        rowptr[0] = 0;
        for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
        free(B);
        return rowptr[n];
    }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = rowptr[i];
        const double *xi = X + (size_t)i * d;
        for (int64_t j = 0; j < n; ++j) {
            const double *xj = X + (size_t)j * d;
            if (j == i || pair_in(h, xi, xj, B + (size_t)i * w, B + (size_t)j * w)) {
                double v = pair_value(h, xi, xj, B + (size_t)i * w, B + (size_t)j * w);
                if (j == i) v = v + h->sigma2;
                col[p] = (int32_t)j;
                if (val) val[p] = v;
                ++p;
            }
        }
    }
    free(B);
    return rowptr[n];
}

/* One row of A by brute force (used to check sampled rows at sizes where the full
 * all-pairs pass is too slow).  cols/vals need room for n entries.  Returns the count. */
int64_t orc_row_brute(int64_t n, const double *X, const orc_hyper *h, int64_t i,
                      int32_t *cols, double *vals)
{
    const int d = h->d;
    double bi[64], bj[64];
    if (point_width(h) > 64) return -1;
    const double *xi = X + (size_t)i * d;
    point_values(h, xi, bi);
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
        const double *xj = X + (size_t)j * d;
        if (h->family == 1 && j != i) point_values(h, xj, bj);
        if (j == i || pair_in(h, xi, xj, bi, bj)) {
            if (h->family != 1 || j == i) point_values(h, xj, bj);
            double v = pair_value(h, xi, xj, bi, bj);
            if (j == i) v = v + h->sigma2;
            cols[c] = (int32_t)j;
            if (vals) vals[c] = v;
            ++c;
        }
    }
    return c;
}

/* Several rows by brute force, rows[0..nrows-1]; row r's entries go to
 * cols[r * n + ...] / vals[r * n + ...] and its count to counts[r]. */
void orc_rows_brute(int64_t n, const double *X, const orc_hyper *h, int64_t nrows,
                    const int64_t *rows, int32_t *cols, double *vals, int64_t *counts)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r)
        counts[r] = orc_row_brute(n, X, h, rows[r], cols + (size_t)r * n,
                                  vals ? vals + (size_t)r * n : NULL);
}

/* ------------------------------------------------------------------------------------ */
/* Assembly from a candidate list.  For large n a spatial search (a library k-d tree,  */
/* queried with a slightly enlarged radius) supplies unordered candidate pairs (i < j);  */
/* the exact FP64 pattern test and the kernel definition then decide and value each     */
/* pair here, so the result is the same set the brute-force pass produces.             */
/*   cand_i, cand_j: ncand pairs with i < j (duplicates not allowed).                  */
/*   First call with col == NULL fills rowptr (n+1) and returns nnz; second call fills */
/*   col/val with columns ascending per row.                                           */
/* ------------------------------------------------------------------------------------ */
static int cmp_col(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_assemble_candidates(int64_t n, const double *X, const orc_hyper *h,
                                int64_t ncand, const int64_t *cand_i, const int64_t *cand_j,
                                int64_t *rowptr, int32_t *col, double *val)
{
    const int d = h->d, w = point_width(h);
    double *B = bump_table(n, X, h);
    if (!B) return -1;
    if (!col) {
        for (int64_t i = 0; i <= n; ++i) rowptr[i] = 0;
        for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = 1;   /* the diagonal */
        for (int64_t p = 0; p < ncand; ++p) {
            int64_t i = cand_i[p], j = cand_j[p];
            if (pair_in(h, X + (size_t)i * d, X + (size_t)j * d, B + (size_t)i * w, B + (size_t)j * w)) {
                rowptr[i + 1] += 1;
                rowptr[j + 1] += 1;
            }
        }
        for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
        free(B);
        return rowptr[n];
    }
    int64_t *fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fillp) { free(B); return -1; }
    for (int64_t i = 0; i < n; ++i) { fillp[i] = rowptr[i] + 1; col[rowptr[i]] = (int32_t)i; }
    for (int64_t p = 0; p < ncand; ++p) {
        int64_t i = cand_i[p], j = cand_j[p];
        if (pair_in(h, X + (size_t)i * d, X + (size_t)j * d, B + (size_t)i * w, B + (size_t)j * w)) {
            col[fillp[i]++] = (int32_t)j;
            col[fillp[j]++] = (int32_t)i;
        }
    }
    free(fillp);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = rowptr[i], e = rowptr[i + 1];
        qsort(col + a, (size_t)(e - a), sizeof(int32_t), cmp_col);
        if (val) {
            const double *xi = X + (size_t)i * d;
            for (int64_t p = a; p < e; ++p) {
                int64_t j = col[p];
                double v = pair_value(h, xi, X + (size_t)j * d, B + (size_t)i * w, B + (size_t)j * w);
                if (j == i) v = v + h->sigma2;
                val[p] = v;
            }
        }
    }
    free(B);
    return rowptr[n];
}

/* Dense A = K + sigma^2 I (n x n, row-major), for the exact small-n path. */
void orc_dense_A(int64_t n, const double *X, const orc_hyper *h, double *A)
{
    const int d = h->d, w = point_width(h);
    double *B = bump_table(n, X, h);
    if (!B) return;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            const double *xi = X + (size_t)i * d, *xj = X + (size_t)j * d;
            double v = 0.0;
            if (j == i || pair_in(h, xi, xj, B + (size_t)i * w, B + (size_t)j * w))
                v = pair_value(h, xi, xj, B + (size_t)i * w, B + (size_t)j * w);
            if (j == i) v = v + h->sigma2;
            A[(size_t)i * n + j] = v;
        }
    free(B);
}

/* Cross-covariance for the posterior of Sec. 3 (Eq. 2): Ks[i * n + j] = k(xs_i, x_j) for
 * test points xs (ns x d) and training points x (n x d), every pair evaluated; the entry is
 * nonzero only inside the support, d2 < r*r (strict), with d2 in the pattern's FP64 order.
 * No noise term: a test point is a new location, never the same index as a training point. */
void orc_cross_K(int64_t ns, const double *Xs, int64_t n, const double *X, const orc_hyper *h, double *Ks)
{
    const int d = h->d, w = point_width(h);
    double *B = bump_table(n, X, h);
    double *Bs = bump_table(ns, Xs, h);
    if (!B || !Bs) { free(B); free(Bs); return; }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < ns; ++i)
        for (int64_t j = 0; j < n; ++j) {
            const double *xi = Xs + (size_t)i * d, *xj = X + (size_t)j * d;
            double v = 0.0;
            if (pair_in(h, xi, xj, Bs + (size_t)i * w, B + (size_t)j * w))
                v = pair_value(h, xi, xj, Bs + (size_t)i * w, B + (size_t)j * w);
            Ks[(size_t)i * n + j] = v;
        }
    free(B);
    free(Bs);
}

/* ------------------------------------------------------------------------------------ */
/* Sparse products and Krylov methods in FP64.                                          */
/* ------------------------------------------------------------------------------------ */

/* Y = M X for an n x n CSR matrix M and k right-hand sides (X, Y: n x k row-major). */
void orc_spmm(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
              int k, const double *Xin, double *Yout)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *y = Yout + (size_t)i * k;
        for (int c = 0; c < k; ++c) y[c] = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double *x = Xin + (size_t)col[p] * k;
            double v = val[p];
            for (int c = 0; c < k; ++c) y[c] = y[c] + v * x[c];
        }
    }
}

/* Column dot products of two n x k matrices.  Rows are summed in fixed chunks of 4096 in
 * row order and the chunk sums are added in chunk order, so the result does not depend on the
 * number of threads. */
static void coldots(int64_t n, int k, const double *A, const double *B, double *out)
{
    const int64_t CH = 4096;
    int64_t nch = (n + CH - 1) / CH;
    double *part = (double *)calloc((size_t)(nch > 0 ? nch : 1) * (size_t)k, sizeof(double));
    for (int c = 0; c < k; ++c) out[c] = 0.0;
    if (!part) return;
    #pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nch; ++b) {
        double *pp = part + (size_t)b * k;
        int64_t e = (b + 1) * CH < n ? (b + 1) * CH : n;
        for (int64_t i = b * CH; i < e; ++i)
            for (int c = 0; c < k; ++c) pp[c] = pp[c] + A[(size_t)i * k + c] * B[(size_t)i * k + c];
    }
    for (int64_t b = 0; b < nch; ++b)
        for (int c = 0; c < k; ++c) out[c] = out[c] + part[(size_t)b * k + c];
    free(part);
}

/*
 * Conjugate gradients (Hestenes & Stiefel) on the SPD CSR matrix M for k independent
 * right-hand sides B (n x k), x0 = 0.  Column c stops updating once
 * |r_c| <= tol * |b_c| or after maxit iterations.  For column c the first kmax step
 * lengths alpha_j and direction coefficients beta_j = rho_{j+1}/rho_j are written to
 * alpha[c*kmax + j], beta[c*kmax + j] (either may be NULL); steps[c] receives the number
 * of iterations the column took.  Returns 0, or 1 if some column hit p^T M p <= 0.
 */
int orc_cg(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
           int k, const double *Bm, double *Xm, double tol, int maxit,
           int kmax, double *alpha, double *beta, int *steps)
{
    size_t nk = (size_t)n * k;
    double *R = (double *)malloc(sizeof(double) * nk);
    double *P = (double *)malloc(sizeof(double) * nk);
    double *Q = (double *)malloc(sizeof(double) * nk);
    double *rho = (double *)malloc(sizeof(double) * k);
    double *bn = (double *)malloc(sizeof(double) * k);
    double *pq = (double *)malloc(sizeof(double) * k);
    double *rr = (double *)malloc(sizeof(double) * k);
    double *bta = (double *)malloc(sizeof(double) * k);
    int *act = (int *)malloc(sizeof(int) * k);
    int status = 0;
    if (!R || !P || !Q || !rho || !bn || !pq || !rr || !bta || !act) { status = -1; goto done; }
    for (size_t e = 0; e < nk; ++e) { Xm[e] = 0.0; R[e] = Bm[e]; P[e] = Bm[e]; }
    coldots(n, k, R, R, rho);
    for (int c = 0; c < k; ++c) {
        bn[c] = sqrt(rho[c]);
        act[c] = !(bn[c] == 0.0);
        if (steps) steps[c] = 0;
    }
    for (int it = 0; it < maxit; ++it) {
        int any = 0;
        for (int c = 0; c < k; ++c)
            if (act[c] && sqrt(rho[c]) <= tol * bn[c]) act[c] = 0;
        for (int c = 0; c < k; ++c) any |= act[c];
        if (!any) break;
        orc_spmm(n, rowptr, col, val, k, P, Q);
        coldots(n, k, P, Q, pq);
        for (int c = 0; c < k; ++c) {
            if (!act[c]) continue;
            if (!(pq[c] > 0.0)) { act[c] = 0; status = 1; continue; }
            pq[c] = rho[c] / pq[c];   /* alpha_c */
        }
        /* x_c += alpha_c p_c ; r_c -= alpha_c q_c */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < k; ++c) {
                if (!act[c]) continue;
                size_t e = (size_t)i * k + c;
                Xm[e] = Xm[e] + pq[c] * P[e];
                R[e] = R[e] - pq[c] * Q[e];
            }
        coldots(n, k, R, R, rr);
        for (int c = 0; c < k; ++c) {
            if (!act[c]) continue;
            bta[c] = rr[c] / rho[c];
            if (alpha && it < kmax) alpha[(size_t)c * kmax + it] = pq[c];
            if (beta && it < kmax) beta[(size_t)c * kmax + it] = bta[c];
        }
        /* p_c = r_c + beta_c p_c */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < k; ++c) {
                if (!act[c]) continue;
                size_t e = (size_t)i * k + c;
                P[e] = R[e] + bta[c] * P[e];
            }
        for (int c = 0; c < k; ++c) {
            if (!act[c]) continue;
            rho[c] = rr[c];
            if (steps) steps[c] = it + 1;
        }
    }
done:
    free(R); free(P); free(Q); free(rho); free(bn); free(pq); free(rr); free(bta); free(act);
    return status;
}

/*
 * Lanczos (no reorthogonalisation) on the symmetric CSR matrix M, k starting vectors
 * Q1 (n x k, each of unit norm), up to `steps` steps.  For column c:
 *   diag[c*steps + j] = alpha_j = q_j^T M q_j, off[c*steps + j] = beta_{j+1} = |w_j|,
 * with w_j = M q_j - alpha_j q_j - beta_j q_{j-1}.  The process stops for a column when
 * beta_{j+1} <= 1e-12 * (the largest |alpha| or |beta| seen so far), keeping the j+1
 * rows computed; nsteps[c] is the order of the tridiagonal T_c.
 */
void orc_lanczos(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                 int k, const double *Q1, int steps, double *diag, double *off, int *nsteps)
{
    size_t nk = (size_t)n * k;
    double *Qp = (double *)calloc(nk, sizeof(double));   /* q_{j-1} */
    double *Qc = (double *)malloc(sizeof(double) * nk);  /* q_j */
    double *W = (double *)malloc(sizeof(double) * nk);
    double *tmp = (double *)malloc(sizeof(double) * k);
    double *bprev = (double *)calloc((size_t)k, sizeof(double));
    double *tnorm = (double *)calloc((size_t)k, sizeof(double));
    int *act = (int *)malloc(sizeof(int) * k);
    if (!Qp || !Qc || !W || !tmp || !bprev || !tnorm || !act) goto done;
    memcpy(Qc, Q1, sizeof(double) * nk);
    for (int c = 0; c < k; ++c) { act[c] = 1; nsteps[c] = 0; }
    for (int j = 0; j < steps; ++j) {
        orc_spmm(n, rowptr, col, val, k, Qc, W);
        coldots(n, k, Qc, W, tmp);
        for (int c = 0; c < k; ++c) {
            if (!act[c]) continue;
            diag[(size_t)c * steps + j] = tmp[c];
            nsteps[c] = j + 1;
            if (fabs(tmp[c]) > tnorm[c]) tnorm[c] = fabs(tmp[c]);
        }
        /* w = M q_j - alpha_j q_j - beta_j q_{j-1} */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < k; ++c) {
                if (!act[c]) continue;
                size_t e = (size_t)i * k + c;
                W[e] = W[e] - tmp[c] * Qc[e] - bprev[c] * Qp[e];
            }
        coldots(n, k, W, W, tmp);
        for (int c = 0; c < k; ++c) {
            if (!act[c]) continue;
            double b = sqrt(tmp[c]);
            off[(size_t)c * steps + j] = b;
            if (b > tnorm[c]) tnorm[c] = b;
            if (j + 1 >= steps || b <= 1e-12 * tnorm[c]) { act[c] = 0; continue; }
            bprev[c] = b;
        }
        /* q_{j+1} = w / beta_{j+1} */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < k; ++c) {
                if (!act[c]) continue;
                size_t e = (size_t)i * k + c;
                Qp[e] = Qc[e];
                Qc[e] = W[e] / bprev[c];
            }
    }
done:
    free(Qp); free(Qc); free(W); free(tmp); free(bprev); free(tnorm); free(act);
}

/* ------------------------------------------------------------------------------------ */
/* Gradient contraction (Sec. 3 LML; the derivative is the standard one,                */
/*   d LML / d theta_p = 1/2 a^T (dA/dtheta_p) a - 1/2 tr(A^{-1} dA/dtheta_p)).         */
/* With W_ij = a_i a_j - T_ij, where T is A^{-1} (exact) or the symmetrised Hutchinson  */
/* estimate T_ij = (1/m) sum_s (U_is V_js + U_js V_is) / 2, the gradient is             */
/*   g_p = 1/2 sum_{(i,j) in pattern} W_ij dA_ij/dtheta_p.                              */
/* theta order: centers (L x d), radii (L), amps (L), r, sigma2; P = L (d + 2) + 2.     */
/* ------------------------------------------------------------------------------------ */

/* dA_ij / dtheta for one stored pair, all P parameters. */
static void pair_grad(const orc_hyper *h, const double *xi, const double *xj, int diag,
                      const double *bi, const double *dbi, const double *bj, const double *dbj,
                      double *g)
{
    const int d = h->d, L = h->L;
    const int P = L * (d + 2) + 2;
    double q = orc_sqdist(d, xi, xj);
    double t = sqrt(q) / h->r;
    double phi = orc_phi(h->kind, d, t);
    double s = 0.0;
    for (int l = 0; l < L; ++l) s = s + bi[l] * bj[l];
    for (int p = 0; p < P; ++p) g[p] = 0.0;
    for (int l = 0; l < L; ++l) {
        for (int k = 0; k < d; ++k)
            g[l * d + k] = phi * (dbi[l * (d + 2) + k] * bj[l] + bi[l] * dbj[l * (d + 2) + k]);
        g[L * d + l] = phi * (dbi[l * (d + 2) + d] * bj[l] + bi[l] * dbj[l * (d + 2) + d]);
        g[L * d + L + l] = phi * (dbi[l * (d + 2) + d + 1] * bj[l] + bi[l] * dbj[l * (d + 2) + d + 1]);
    }
    /* d phi(|xi-xj|/r) / d r = phi'(t) * (-t / r) */
    g[P - 2] = (s + h->w0) * orc_dphi(h->kind, d, t) * (-t / h->r);
    g[P - 1] = diag ? 1.0 : 0.0;
}

/* Family 1 (Eq. 6): per-point quantities for the gradient: s, lambda (d), psi (L) and
 * d psi_l / d(c_l, rho_l) (L x (d + 1)). */
typedef struct { double s, lam[4], psi[32], dpsi[32 * 5]; } wc_pt;

static void wc_point_grad(const orc_hyper *h, const double *x, wc_pt *p)
{
    const int d = h->d, L = h->L;
    double v[5];
    wc_point(h, x, v);
    p->s = v[0];
    for (int k = 0; k < d; ++k) p->lam[k] = v[1 + k];
    for (int l = 0; l < L; ++l) {
        double s;
        p->psi[l] = wc_psi(h, l, x, &s);
        double *g = p->dpsi + (size_t)l * (d + 1);
        if (s < 1.0) {
            double u = 1.0 - s, rho = h->radii[l];
            double dpds = -3.0 * u * u;
            const double *c = h->centers + (size_t)l * d;
            for (int k = 0; k < d; ++k) g[k] = dpds * (-2.0 * (x[k] - c[k]) / (rho * rho));
            g[d] = dpds * (-2.0 * s / rho);
        } else {
            for (int k = 0; k <= d; ++k) g[k] = 0.0;
        }
    }
}

/* dA_ij / dtheta for one stored pair of the family-1 kernel; theta = [centers (L x d),
 * radii (L), amps (L), G (L x d), ell (d), w0, r0, sigma2]. */
static void pair_grad_wc(const orc_hyper *h, const double *xi, const double *xj, int diag, const wc_pt *pi,
                         const wc_pt *pj, double *g)
{
    const int d = h->d, L = h->L;
    const int P = L * (2 * d + 2) + d + 3;
    const int oC = 0, oR = L * d, oA = L * d + L, oG = L * d + 2 * L, oE = L * (2 * d + 2), oW = oE + d;
    for (int p = 0; p < P; ++p) g[p] = 0.0;
    double ds[2], dl[2][4], dr0 = 0.0;
    if (diag) {
        /* k_ii = s_i^2 whatever lambda and r0: only s moves it */
        ds[0] = pi->s;
        ds[1] = pi->s;
        for (int k = 0; k < d; ++k) dl[0][k] = dl[1][k] = 0.0;
        g[P - 1] = 1.0;
    } else {
        double q = orc_wc_q(d, xi, xj, pi->lam, pj->lam);
        double t = sqrt(q) / h->r;
        double phi = orc_phi(h->kind, d, t);
        double pref = 1.0;
        for (int k = 0; k < d; ++k)
            pref = pref * sqrt(sqrt(pi->lam[k] * pj->lam[k])) / sqrt((pi->lam[k] + pj->lam[k]) * 0.5);
        double dphidq = orc_dphi_over_t(h->kind, d, t) / (2.0 * h->r * h->r);
        double ss = pi->s * pj->s;
        ds[0] = pj->s * pref * phi;
        ds[1] = pi->s * pref * phi;
        for (int k = 0; k < d; ++k) {
            double m = (pi->lam[k] + pj->lam[k]) * 0.5;
            double dk = xi[k] - xj[k];
            double dq = -(dk * dk) / (2.0 * m * m);      /* dQ / d lambda_{i or j, k} */
            dl[0][k] = ss * (pref * phi * (1.0 / (4.0 * pi->lam[k]) - 1.0 / (4.0 * m)) + pref * dphidq * dq);
            dl[1][k] = ss * (pref * phi * (1.0 / (4.0 * pj->lam[k]) - 1.0 / (4.0 * m)) + pref * dphidq * dq);
        }
        dr0 = ss * pref * orc_dphi(h->kind, d, t) * (-t / h->r);
    }
    const wc_pt *side[2] = {pi, pj};
    for (int e = 0; e < 2; ++e) {
        const wc_pt *pp = side[e];
        for (int l = 0; l < L; ++l) {
            /* through psi_l: s gets a_l psi_l, lambda_k gets G_lk psi_l */
            double w = ds[e] * h->amps[l];
            for (int k = 0; k < d; ++k) w = w + dl[e][k] * h->G[(size_t)l * d + k];
            for (int k = 0; k < d; ++k) g[oC + l * d + k] += w * pp->dpsi[(size_t)l * (d + 1) + k];
            g[oR + l] += w * pp->dpsi[(size_t)l * (d + 1) + d];
            g[oA + l] += ds[e] * pp->psi[l];
            for (int k = 0; k < d; ++k) g[oG + l * d + k] += dl[e][k] * pp->psi[l];
        }
        for (int k = 0; k < d; ++k) g[oE + k] += dl[e][k] * 2.0 * h->ell[k];
        g[oW] += ds[e];
    }
    g[oW + 1] = dr0;
}

/* dA_ij / dtheta for one stored pair of the far-field kernel (family 2); theta = [centers
 * (L x d), radii (L), amps (L), lc, w0, r, sigma2]. */
static void pair_grad_ff(const orc_hyper *h, const double *xi, const double *xj, int diag, const double *bi,
                         const double *dbi, const double *bj, const double *dbj, double *g)
{
    const int d = h->d, L = h->L;
    const int P = L * (d + 2) + 4;
    double q = orc_sqdist(d, xi, xj);
    double kap = ff_kappa(h, q);
    int in_ball = diag || q < h->r * h->r;
    double t = sqrt(q) / h->r;
    double sb = 0.0;
    for (int l = 0; l < L; ++l) sb = sb + bi[l] * bj[l];
    for (int p = 0; p < P; ++p) g[p] = 0.0;
    for (int l = 0; l < L; ++l) {
        for (int k = 0; k < d; ++k)
            g[l * d + k] = kap * (dbi[l * (d + 2) + k] * bj[l] + bi[l] * dbj[l * (d + 2) + k]);
        g[L * d + l] = kap * (dbi[l * (d + 2) + d] * bj[l] + bi[l] * dbj[l * (d + 2) + d]);
        g[L * d + L + l] = kap * (dbi[l * (d + 2) + d + 1] * bj[l] + bi[l] * dbj[l * (d + 2) + d + 1]);
    }
    double lc = h->ell[0];
    g[P - 4] = sb * kap * q / (lc * lc * lc);                       /* d kappa / d lc */
    g[P - 3] = in_ball ? orc_phi(h->kind, d, t) : 0.0;             /* d / d w0 */
    g[P - 2] = in_ball ? h->w0 * orc_dphi(h->kind, d, t) * (-t / h->r) : 0.0;
    g[P - 1] = diag ? 1.0 : 0.0;
}

/*
 * grad[P] = 1/2 sum over stored (i, j) of W_ij dA_ij.  The pattern is given in CSR
 * (rowptr, col; original index order).  If Wd (n x n) is non-NULL, W_ij = a_i a_j - Wd_ij;
 * otherwise W_ij = a_i a_j - (1/m) sum_s (U_is V_js + U_js V_is) / 2 with U, V n x m.
 * Row partial sums are added in row order (deterministic).
 */
static double pair_w(int64_t n, int64_t i, int64_t j, const double *a, int m, const double *U, const double *V,
                     const double *Wd)
{
    if (Wd) return a[i] * a[j] - Wd[(size_t)i * n + j];
    double tr = 0.0;
    for (int s = 0; s < m; ++s)
        tr = tr + 0.5 * (U[(size_t)i * m + s] * V[(size_t)j * m + s] + U[(size_t)j * m + s] * V[(size_t)i * m + s]);
    return a[i] * a[j] - tr / (double)m;
}

static int grad_contract_wc(int64_t n, const int64_t *rowptr, const int32_t *col, const double *X,
                            const orc_hyper *h, const double *a, int m, const double *U, const double *V,
                            const double *Wd, double *grad)
{
    const int d = h->d, L = h->L;
    const int P = L * (2 * d + 2) + d + 3;
    const int64_t chunk = 4096;
    if (L > 32 || P > 512) return -1;
    wc_pt *pts = (wc_pt *)malloc(sizeof(wc_pt) * (size_t)(n > 0 ? n : 1));
    double *rowg = (double *)malloc(sizeof(double) * (size_t)chunk * P);
    if (!pts || !rowg) { free(pts); free(rowg); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) wc_point_grad(h, X + (size_t)i * d, pts + i);
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    for (int64_t i0 = 0; i0 < n; i0 += chunk) {
        int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
        #pragma omp parallel for schedule(dynamic, 32)
        for (int64_t i = i0; i < i1; ++i) {
            double g[512];
            double *acc = rowg + (size_t)(i - i0) * P;
            for (int p = 0; p < P; ++p) acc[p] = 0.0;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                int64_t j = col[e];
                double w = pair_w(n, i, j, a, m, U, V, Wd);
                pair_grad_wc(h, X + (size_t)i * d, X + (size_t)j * d, j == i, pts + i, pts + j, g);
                for (int p = 0; p < P; ++p) acc[p] = acc[p] + 0.5 * w * g[p];
            }
        }
        for (int64_t i = i0; i < i1; ++i)
            for (int p = 0; p < P; ++p) grad[p] = grad[p] + rowg[(size_t)(i - i0) * P + p];
    }
    free(pts);
    free(rowg);
    return 0;
}

int orc_grad_contract(int64_t n, const int64_t *rowptr, const int32_t *col, const double *X,
                      const orc_hyper *h, const double *a, int m, const double *U,
                      const double *V, const double *Wd, double *grad)
{
    const int d = h->d, L = h->L;
    if (h->family == 1) return grad_contract_wc(n, rowptr, col, X, h, a, m, U, V, Wd, grad);
    const int P = h->family == 2 ? L * (d + 2) + 4 : L * (d + 2) + 2;
    const int64_t chunk = 4096;
    double *B = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(L > 0 ? L : 1));
    double *dB = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(L * (d + 2) > 0 ? L * (d + 2) : 1));
    double *rowg = (double *)malloc(sizeof(double) * (size_t)chunk * P);
    if (!B || !dB || !rowg) { free(B); free(dB); free(rowg); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        orc_bumps(h, X + (size_t)i * d, B + (size_t)i * L, dB + (size_t)i * L * (d + 2));
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    for (int64_t i0 = 0; i0 < n; i0 += chunk) {
        int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
        #pragma omp parallel for schedule(dynamic, 32)
        for (int64_t i = i0; i < i1; ++i) {
            double g[512];
            double *acc = rowg + (size_t)(i - i0) * P;
            for (int p = 0; p < P; ++p) acc[p] = 0.0;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                int64_t j = col[e];
                double w;
                if (Wd) {
                    w = a[i] * a[j] - Wd[(size_t)i * n + j];
                } else {
                    double tr = 0.0;
                    for (int s = 0; s < m; ++s)
                        tr = tr + 0.5 * (U[(size_t)i * m + s] * V[(size_t)j * m + s] +
                                         U[(size_t)j * m + s] * V[(size_t)i * m + s]);
                    w = a[i] * a[j] - tr / (double)m;
                }
                if (h->family == 2)
                    pair_grad_ff(h, X + (size_t)i * d, X + (size_t)j * d, j == i,
                                 B + (size_t)i * L, dB + (size_t)i * L * (d + 2),
                                 B + (size_t)j * L, dB + (size_t)j * L * (d + 2), g);
                else
                    pair_grad(h, X + (size_t)i * d, X + (size_t)j * d, j == i,
                              B + (size_t)i * L, dB + (size_t)i * L * (d + 2),
                              B + (size_t)j * L, dB + (size_t)j * L * (d + 2), g);
                for (int p = 0; p < P; ++p) acc[p] = acc[p] + 0.5 * w * g[p];
            }
        }
        for (int64_t i = i0; i < i1; ++i)
            for (int p = 0; p < P; ++p) grad[p] = grad[p] + rowg[(size_t)(i - i0) * P + p];
    }
    free(B); free(dB); free(rowg);
    return 0;
}

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
