/*
 * dade_oracle.c -- plain FP64 CPU oracle for DADE inside an IVF scan and
 * inside HNSW's layer-0 beam search (HNSW*).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code with
 * the CUDA library: nothing here is included by, linked into or generated for
 * the GPU path, and it includes nothing of it.
 *
 * Every routine follows the paper (Deng et al., "Efficient Data-aware Distance
 * Comparison Operations for High-Dimensional Approximate Nearest Neighbor
 * Search") step by step, in double precision, with no blocking or reordering
 * beyond what the cited definition states.  Sums run in index order.
 * OpenMP is used only across independent outputs (rows of the covariance,
 * base points in an assignment step, queries), never inside one sum.
 *
 * Notation: D dimensions, W = [w_1..w_D] the PCA basis (column k of W is w_k),
 * lambda_1 >= ... >= lambda_D, Lambda_d = sum_{k<=d} lambda_k,
 * P_d(q,o) = sum_{k<=d} (q'_k - o'_k)^2 in the rotated space, r the current
 * K-th nearest distance.  Row-major arrays throughout.
 *
 * The beam search also runs in the FP32 arithmetic of the paper's scalar
 * implementation (dco_f32): the decisions of a graph search steer which
 * objects are visited, so the CUDA path is compared with the oracle making
 * them in the same precision; that mode is pinned to the FP64 one.
 *
 * Parity status: every routine is pinned by the CPU tests (closed forms,
 * library routines on special cases, brute force on tiny inputs, statistical
 * checks).  The recall level of the whole search has no printed value in the
 * paper and is reported, not pinned ("parity unpinned" for absolute recall).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_API __attribute__((visibility("default")))

OR_API void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

OR_API int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Section 3.2, Eq. 10-12: PCA of E[X X^T] over all data objects, after      */
/* centring (Lemma 1 makes the mean free: distances are unchanged).          */
/* ------------------------------------------------------------------------ */

/* mu_j = (1/n) sum_i x_ij ;  C_jk = (1/n) sum_i (x_ij - mu_j)(x_ik - mu_k). */
OR_API void or_mean_cov(const float *X, int64_t n, int d, double *mu, double *C)
{
    for (int j = 0; j < d; ++j) mu[j] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j) mu[j] += (double)X[i * d + j];
    for (int j = 0; j < d; ++j) mu[j] /= (double)n;

    /* Each entry sums over i in order.  The rows of X are visited in blocks
     * that every thread reads while they are in cache (one covariance row j
     * per thread within a block), so X streams from memory about once. */
    for (int64_t t = 0; t < (int64_t)d * d; ++t) C[t] = 0.0;
    const int64_t blk = 2048;
    #pragma omp parallel
    for (int64_t i0 = 0; i0 < n; i0 += blk) {
        const int64_t i1 = i0 + blk < n ? i0 + blk : n;
        #pragma omp for schedule(dynamic, 1)
        for (int j = 0; j < d; ++j) {
            double *row = C + (int64_t)j * d;
            for (int64_t i = i0; i < i1; ++i) {
                const float *x = X + i * d;
                double yj = (double)x[j] - mu[j];
                for (int k = j; k < d; ++k) row[k] += yj * ((double)x[k] - mu[k]);
            }
        }
    }
    for (int j = 0; j < d; ++j)
        for (int k = j; k < d; ++k) C[(int64_t)j * d + k] /= (double)n;
    for (int j = 0; j < d; ++j)
        for (int k = 0; k < j; ++k) C[(int64_t)j * d + k] = C[(int64_t)k * d + j];
}

/*
 * Cyclic Jacobi eigendecomposition of the symmetric d x d matrix A (Jacobi's
 * method: repeated plane rotations that zero one off-diagonal entry at a
 * time).  On return the eigenvalues are in lam (descending, Eq. 11: lambda_k
 * is the k-th largest) and column k of V is the matching unit eigenvector w_k.
 * A is overwritten.  Returns the number of sweeps, or -1 if not converged.
 */
OR_API int or_jacobi_eig(double *A, int d, double *lam, double *V)
{
    /* the eigenproblem of a symmetric matrix: take (A + A^T) / 2 (a no-op on
     * the exactly symmetric covariance of or_mean_cov) */
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j) {
            double m = 0.5 * (A[(int64_t)i * d + j] + A[(int64_t)j * d + i]);
            A[(int64_t)i * d + j] = m;
            A[(int64_t)j * d + i] = m;
        }
    double fro = 0.0;
    for (int64_t t = 0; t < (int64_t)d * d; ++t) fro += A[t] * A[t];
    fro = sqrt(fro);
    /* VT = V^T: row k of VT is eigenvector column k, so the updates of two
     * eigenvector columns touch two contiguous rows */
    double *VT = (double *)malloc(sizeof(double) * (size_t)d * d);
    if (!VT) return -1;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) VT[(int64_t)i * d + j] = (i == j) ? 1.0 : 0.0;

    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) off += 2.0 * A[(int64_t)p * d + q] * A[(int64_t)p * d + q];
        if (sqrt(off) <= 1e-14 * fro || fro == 0.0) break;
        for (int p = 0; p < d - 1; ++p) {
            for (int q = p + 1; q < d; ++q) {
                double *Ap = A + (int64_t)p * d, *Aq = A + (int64_t)q * d;
                double apq = Ap[q];
                if (apq == 0.0) continue;
                double app = Ap[p], aqq = Aq[q];
                /* rotation angle that annihilates a_pq */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J.  A stays symmetric, so for k outside {p, q} the new
                 * rows p, q and columns p, q hold the same values: compute them on
                 * the rows, mirror them into the columns */
                for (int k = 0; k < d; ++k) {
                    if (k == p || k == q) continue;
                    double apk = Ap[k], aqk = Aq[k];
                    double np = c * apk - s * aqk, nq = s * apk + c * aqk;
                    Ap[k] = np;
                    Aq[k] = nq;
                    A[(int64_t)k * d + p] = np;
                    A[(int64_t)k * d + q] = nq;
                }
                /* the 2 x 2 block: A J (columns p, q), then J^T (rows p, q) */
                double bpp = c * app - s * apq, bpq = s * app + c * apq;
                double bqp = c * apq - s * aqq, bqq = s * apq + c * aqq;
                Ap[p] = c * bpp - s * bqp;
                Aq[q] = s * bpq + c * bqq;
                Ap[q] = 0.0;
                Aq[p] = 0.0;
                double *Vp = VT + (int64_t)p * d, *Vq = VT + (int64_t)q * d;
                for (int k = 0; k < d; ++k) {      /* V <- V J */
                    double vkp = Vp[k], vkq = Vq[k];
                    Vp[k] = c * vkp - s * vkq;
                    Vq[k] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < d; ++i) lam[i] = A[(int64_t)i * d + i];
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) V[(int64_t)k * d + i] = VT[(int64_t)i * d + k];
    free(VT);
    /* order eigenpairs by descending eigenvalue (selection sort: plain) */
    for (int i = 0; i < d; ++i) {
        int best = i;
        for (int j = i + 1; j < d; ++j) if (lam[j] > lam[best]) best = j;
        if (best != i) {
            double tl = lam[i]; lam[i] = lam[best]; lam[best] = tl;
            for (int k = 0; k < d; ++k) {
                double tv = V[(int64_t)k * d + i];
                V[(int64_t)k * d + i] = V[(int64_t)k * d + best];
                V[(int64_t)k * d + best] = tv;
            }
        }
    }
    return sweep < 100 ? sweep : -1;
}

/* PCA: mean, covariance and its eigendecomposition (Eq. 11, Eq. 12). */
OR_API int or_pca(const float *X, int64_t n, int d, double *mu, double *W, double *lam)
{
    double *C = (double *)malloc(sizeof(double) * (size_t)d * d);
    if (!C) return -1;
    or_mean_cov(X, n, d, mu, C);
    int s = or_jacobi_eig(C, d, lam, W);
    free(C);
    return s;
}

/* Rotation x' = W^T (x - mu): out_ik = sum_j W_jk (x_ij - mu_j)  (Lemma 1). */
OR_API void or_rotate(const float *X, int64_t n, int d, const double *mu, const double *W, double *out)
{
    /* every out_ik sums over j in order; the j loop is outermost so that W is
     * read a row at a time */
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const float *x = X + i * d;
        double *o = out + i * d;
        for (int k = 0; k < d; ++k) o[k] = 0.0;
        for (int j = 0; j < d; ++j) {
            const double y = (double)x[j] - mu[j];
            const double *w = W + (int64_t)j * d;
            for (int k = 0; k < d; ++k) o[k] += w[k] * y;
        }
    }
}

/* Squared Euclidean distance between two FP64 vectors, summed in order. */
static double sqdist(const double *a, const double *b, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) { double t = a[k] - b[k]; s += t * t; }
    return s;
}

/* ------------------------------------------------------------------------ */
/* IVF (Section 3.4): k-means centroids, inverted lists, probing.            */
/* ------------------------------------------------------------------------ */

/* Argmin of one row of squared distances; ties go to the lower centroid
 * index.  *gap gets the relative gap between the best and second best. */
static int argmin_row(const double *row, int nc, double *gap)
{
    int best = 0;
    double b1 = INFINITY, b2 = INFINITY;
    for (int c = 0; c < nc; ++c) {
        double t = row[c];
        if (t < b1) { b2 = b1; b1 = t; best = c; }
        else if (t < b2) b2 = t;
    }
    if (gap) *gap = (b2 - b1) / (b1 > 0.0 ? b1 : 1.0);
    return best;
}

/* Squared distances from points X[0..np) to every centroid.  Each distance
 * is the sum over k of (x_k - c_k)^2 in index order; the loops run over the
 * centroids innermost (centroids stored transposed, CT[k * nc + c]) so that
 * many independent sums advance together. */
#define OR_PB 8
static void block_dists(const double *X, int np, int d, const double *CT, int nc, double *acc)
{
    for (int64_t t = 0; t < (int64_t)np * nc; ++t) acc[t] = 0.0;
    for (int k = 0; k < d; ++k) {
        const double *ct = CT + (int64_t)k * nc;
        for (int b = 0; b < np; ++b) {
            const double xk = X[(int64_t)b * d + k];
            double *a = acc + (int64_t)b * nc;
            for (int c = 0; c < nc; ++c) { double t = xk - ct[c]; a[c] += t * t; }
        }
    }
}

/* assign[i] = nearest centroid of every point (ties to the lower index);
 * returns the smallest relative best/second-best gap. */
static double assign_all(const double *Xr, int64_t n, int d, const double *cent, int nc, int32_t *assign)
{
    double *CT = (double *)malloc(sizeof(double) * (size_t)nc * d);
    for (int c = 0; c < nc; ++c)
        for (int k = 0; k < d; ++k) CT[(int64_t)k * nc + c] = cent[(int64_t)c * d + k];
    double g = INFINITY;
    #pragma omp parallel reduction(min:g)
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)OR_PB * nc);
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i0 = 0; i0 < n; i0 += OR_PB) {
            int np = (int)(n - i0 < OR_PB ? n - i0 : OR_PB);
            block_dists(Xr + i0 * d, np, d, CT, nc, acc);
            for (int b = 0; b < np; ++b) {
                double gi;
                assign[i0 + b] = argmin_row(acc + (int64_t)b * nc, nc, &gi);
                if (gi < g) g = gi;
            }
        }
        free(acc);
    }
    free(CT);
    return g;
}

/*
 * Lloyd k-means: centroids start at the given base points; each iteration
 * assigns every point to its nearest centroid and moves every centroid to
 * the mean of its members (an empty cluster keeps its previous centroid).
 * obj[it] = sum of squared distances in iteration it's assignment step.
 * min_gap = smallest relative best/second-best gap seen (near-tie indicator).
 * assign holds the last iteration's assignment (before the final update).
 */
OR_API void or_kmeans(const double *Xr, int64_t n, int d, int nc, const int64_t *init, int iters,
                      double *cent, int32_t *assign, double *obj, double *min_gap)
{
    for (int c = 0; c < nc; ++c)
        memcpy(cent + (int64_t)c * d, Xr + init[c] * d, sizeof(double) * d);
    double *sum = (double *)malloc(sizeof(double) * (size_t)nc * d);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    double gmin = INFINITY;
    for (int it = 0; it < iters; ++it) {
        double o = 0.0;
        double g = assign_all(Xr, n, d, cent, nc, assign);
        for (int64_t i = 0; i < n; ++i) o += sqdist(Xr + i * d, cent + (int64_t)assign[i] * d, d);
        if (obj) obj[it] = o;
        if (g < gmin) gmin = g;
        memset(sum, 0, sizeof(double) * (size_t)nc * d);
        memset(cnt, 0, sizeof(int64_t) * (size_t)nc);
        for (int64_t i = 0; i < n; ++i) {
            int c = assign[i];
            cnt[c] += 1;
            for (int k = 0; k < d; ++k) sum[(int64_t)c * d + k] += Xr[i * d + k];
        }
        for (int c = 0; c < nc; ++c)
            if (cnt[c] > 0)
                for (int k = 0; k < d; ++k) cent[(int64_t)c * d + k] = sum[(int64_t)c * d + k] / (double)cnt[c];
    }
    if (min_gap) *min_gap = gmin;
    free(sum);
    free(cnt);
}

/* Inverted lists: every point goes to its nearest centroid (ties to the lower
 * index).  Returns the smallest relative best/second-best gap. */
OR_API double or_assign(const double *Xr, int64_t n, int d, const double *cent, int nc, int32_t *assign)
{
    return assign_all(Xr, n, d, cent, nc, assign);
}

/* Centroid of every list = mean of its members; an empty list gets zeros. */
OR_API void or_list_means(const double *Xr, int64_t n, int d, const int32_t *assign, int nc, double *cent)
{
    int64_t *cnt = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
    memset(cent, 0, sizeof(double) * (size_t)nc * d);
    for (int64_t i = 0; i < n; ++i) {
        cnt[assign[i]] += 1;
        for (int k = 0; k < d; ++k) cent[(int64_t)assign[i] * d + k] += Xr[i * d + k];
    }
    for (int c = 0; c < nc; ++c)
        if (cnt[c] > 0)
            for (int k = 0; k < d; ++k) cent[(int64_t)c * d + k] /= (double)cnt[c];
    free(cnt);
}

typedef struct { double key; int64_t id; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static int dbl_cmp(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static int near_tie(double a, double b, double tol)
{
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    return fabs(a - b) <= tol * m;
}

/* Probe: the nprobe centroids nearest to each query, ordered by (distance,
 * centroid id).  tie[q] = 1 when two of the first nprobe+1 centroid distances
 * are within tol of each other (the order could flip at lower precision). */
OR_API void or_probe(const double *Qr, int64_t nq, int d, const double *cent, int nc, int nprobe,
                     int32_t *probe, int32_t *tie, double tol)
{
    #pragma omp parallel
    {
        kv_t *buf = (kv_t *)malloc(sizeof(kv_t) * (size_t)nc);
        #pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < nq; ++q) {
            for (int c = 0; c < nc; ++c) {
                buf[c].key = sqdist(Qr + q * d, cent + (int64_t)c * d, d);
                buf[c].id = c;
            }
            qsort(buf, (size_t)nc, sizeof(kv_t), kv_cmp);
            int t = 0;
            for (int j = 0; j < nprobe; ++j) {
                probe[q * nprobe + j] = (int32_t)buf[j].id;
                if (j + 1 < nc && near_tie(buf[j].key, buf[j + 1].key, tol)) t = 1;
            }
            if (tie) tie[q] = t;
        }
        free(buf);
    }
}

/* ------------------------------------------------------------------------ */
/* Section 3.3, Eq. 14: epsilon_d from uniformly sampled pairs of objects.   */
/* ------------------------------------------------------------------------ */

/*
 * For each pair (i, j) with nonzero distance, and each d in dlist,
 *   rho_d = dis'_d / dis = sqrt( Lambda_D / Lambda_d * P_d(o_i, o_j) / P_D(o_i, o_j) ),
 * the ratio of the Eq. 13 estimate to the exact distance.  rho is written
 * sorted ascending per d: rho[t * m_kept + s].  Pairs with zero distance are
 * dropped (the ratio is undefined).  Returns m_kept.
 */
OR_API int64_t or_eps_sample(const double *Xr, int64_t n, int d, const double *lam,
                             const int64_t *pairs, int64_t m, const int32_t *dlist, int nd, double *rho)
{
    (void)n;
    double LD = 0.0;
    for (int k = 0; k < d; ++k) LD += lam[k];
    double *Pd = (double *)malloc(sizeof(double) * (size_t)d);
    int64_t kept = 0;
    for (int64_t s = 0; s < m; ++s) {
        const double *a = Xr + pairs[2 * s] * d, *b = Xr + pairs[2 * s + 1] * d;
        double acc = 0.0;
        for (int k = 0; k < d; ++k) { double t = a[k] - b[k]; acc += t * t; Pd[k] = acc; }
        double PD = acc;
        if (!(PD > 0.0)) continue;
        for (int t = 0; t < nd; ++t) {
            int dd = dlist[t];
            double Ld = 0.0;
            for (int k = 0; k < dd; ++k) Ld += lam[k];
            rho[(int64_t)t * m + kept] = sqrt(LD / Ld * Pd[dd - 1] / PD);
        }
        ++kept;
    }
    free(Pd);
    for (int t = 0; t < nd; ++t) qsort(rho + (int64_t)t * m, (size_t)kept, sizeof(double), dbl_cmp);
    return kept;
}

/*
 * epsilon_d for significance level P_s = alpha (Eq. 14): the threshold that
 * rho_d - 1 exceeds with probability alpha, estimated from the sorted sample
 * by the higher order statistic, eps = rho_(ceil((1 - alpha) M)) - 1 (1-based),
 * so that at most a fraction alpha of the sample lies above it.
 */
OR_API double or_eps_quantile(const double *rho_sorted, int64_t m, double alpha)
{
    int64_t idx = (int64_t)ceil((1.0 - alpha) * (double)m);
    if (idx < 1) idx = 1;
    if (idx > m) idx = m;
    return rho_sorted[idx - 1] - 1.0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Section 3.4) with the hypothesis test of Section 3.3.        */
/* ------------------------------------------------------------------------ */

/*
 * One DCO.  q, o: rotated vectors (D dims).  r: the current K-th distance
 * (+inf while fewer than K are held), r2 = r^2 as stored.  Lam[d] = Lambda_d
 * (Lam[0] = 0).  eps[d] = epsilon_d for the tested d.  prune = 0 gives
 * FDScanning (no test before d = D).
 *   d <- 0; while d < D: d <- min(d + delta_d, D);
 *     dis' = sqrt(Lambda_D / Lambda_d * P_d)                      (Eq. 13)
 *     d < D : reject H0 (prune, return 0) iff dis' > (1 + eps_d) r (Section 3.3)
 *     d = D : dis' is the exact distance; accept iff dis <= r      (Definition 1)
 * Returns 1 on accept with *dist2 = P_D.  *dims = dimensions used.
 * *tie |= 1 when a test at d < D had its two sides within tol (relative, on
 * the squared values), |= 2 when the final compare did.
 */
/* Eq. 13 applied to one pair: the squared estimate dis'^2 = Lambda_D / Lambda_d * P_d. */
static double estimate_sq(double Pd, const double *Lam, int D, int d)
{
    return Lam[D] / Lam[d] * Pd;
}

static int dco(const double *q, const double *o, int D, int delta_d, double r, double r2,
               const double *Lam, const double *eps, int prune, double tol,
               double *dist2, int *dims, int *tie)
{
    int d = 0;
    double P = 0.0;
    while (d < D) {
        int dn = d + delta_d;
        if (dn > D) dn = D;
        for (int k = d; k < dn; ++k) { double t = q[k] - o[k]; P += t * t; }
        d = dn;
        if (d < D) {
            if (!prune) continue;
            double est = sqrt(estimate_sq(P, Lam, D, d));
            double bound = (1.0 + eps[d]) * r;
            if (isfinite(r) && near_tie(est * est, bound * bound, tol)) *tie |= 1;
            if (est > bound) { *dims = d; return 0; }
        } else {
            *dims = D;
            *dist2 = P;
            if (isfinite(r2) && near_tie(P, r2, tol)) *tie |= 2;
            return P <= r2;
        }
    }
    *dims = D;
    *dist2 = P;
    return P <= r2;
}

static double *prefix_lambda(const double *lam, int D)
{
    double *Lam = (double *)malloc(sizeof(double) * (size_t)(D + 1));
    Lam[0] = 0.0;
    for (int k = 0; k < D; ++k) Lam[k + 1] = Lam[k] + lam[k];
    return Lam;
}

/* The squared estimate of Eq. 13 for one pair from its first d dimensions. */
OR_API double or_estimate_sq(const double *q, const double *o, int D, int d, const double *lam)
{
    double *Lam = prefix_lambda(lam, D);
    double P = 0.0;
    for (int k = 0; k < d; ++k) { double t = q[k] - o[k]; P += t * t; }
    double e = estimate_sq(P, Lam, D, d);
    free(Lam);
    return e;
}

/* One DCO (Algorithm 1) for one pair; r is the threshold distance (+inf
 * allowed).  Returns 1 on accept; *dist2 gets P_D when accepted; *dims the
 * dimensions used; *tie the near-tie bits of dco(). */
OR_API int or_dco(const double *q, const double *o, int D, int delta_d, double r, const double *lam,
                  const double *eps, int prune, double tol, double *dist2, int *dims, int *tie)
{
    double *Lam = prefix_lambda(lam, D);
    *tie = 0;
    *dist2 = INFINITY;
    int acc = dco(q, o, D, delta_d, r, r * r, Lam, eps, prune, tol, dist2, dims, tie);
    free(Lam);
    return acc;
}

/*
 * IVF search with DADE DCOs (Section 3.4): probe the nprobe nearest lists,
 * scan their members keeping the K nearest (a max-heap in the paper; here a
 * sorted array with the same content), and run one DCO per candidate against
 * the current K-th distance.
 *
 * Candidate order: probe order, then ascending base id within a list.
 * Threshold schedule: candidates form consecutive epochs, and every candidate
 * of an epoch is tested against r taken after all earlier epochs:
 *   schedule 0  SEQUENTIAL      one candidate per epoch (the paper's order);
 *   schedule 1  TILE(tile)      up to `tile` consecutive members of one list;
 *   schedule 2  PROBE_ROUNDS    one whole list per epoch;
 *   schedule 3  ROW_ROUNDS      epoch e holds rows [R_e, R_{e+1}) of every
 *                               probed list (probe order, then row), with
 *                               R_0 = 0, R_1 = tile, R_{e+1} = 2 R_e: every
 *                               list advances by the same rows per epoch, the
 *                               epochs doubling, until the longest probed list
 *                               is done.  Epoch 0 runs with r = +inf.
 * With schedule 1 and lag L > 0, tile t (tiles numbered over the query's
 * whole scan) is tested against r taken after tiles 0..t-1-L only: the
 * threshold of a pipeline that keeps L later tiles in flight.  L = 0 is the
 * plain tile schedule.
 * With seed S > 0 (seeded schedule, schedules 0-2), the first S probed lists
 * run as above and every candidate of the later lists is tested against r
 * frozen at its value after those S lists (a stale r that is the same for all
 * of them); accepted candidates still enter the K nearest.  S >= nprobe is
 * the plain schedule.
 * bias: every decision of the epoch uses r^2 (1 + bias) in place of r^2, both
 * the test at d < D and the final compare.  bias = 0 is the method; runs at
 * bias = -b and +b move every decision within a relative b of its threshold
 * towards pruning and towards keeping, which brackets what a computation at
 * lower precision (error below b) can decide.
 * Results are ordered by (squared distance, id); missing slots are (-1, +inf).
 * eps == NULL runs FDScanning.  eps is indexed by d (eps[d], d < D).
 * stats (nq x 4, may be NULL): candidates, sum of dims used, accepted, pruned.
 * flags (nq, may be NULL): 1|2 test near-ties (see dco), 4 near-tie between
 * the final K-th result and the best accepted candidate that did not stay
 * (a candidate pushed to place K+1 of a merge already has K better ones and
 * can never return, so only the final boundary can change the result),
 * 8 near-tie in the probe order.
 */
#define OR_PEND 4096   /* accepted candidates held before a merge into the K nearest */

/* Merge the npend pending results behind the ntop kept ones into the K
 * nearest by (distance, id).  Within one epoch the threshold is fixed, so
 * merging part of an epoch's results early decides nothing differently. */
static void merge_pending(kv_t *buf, int *ntop, int *npend, int K, double *dropped)
{
    if (*npend == 0) return;
    int u = *ntop + *npend;
    qsort(buf, (size_t)u, sizeof(kv_t), kv_cmp);
    if (u > K && buf[K].key < *dropped) *dropped = buf[K].key;
    *ntop = u < K ? u : K;
    *npend = 0;
}

OR_API int or_search(const double *Xr, int64_t n, int D, const int32_t *assign, int nc,
                     const double *cent, const double *lam, const double *Qr, int64_t nq,
                     int K, int nprobe, int delta_d, const double *eps, int schedule, int tile, int lag,
                     int seed, double tol, double bias, int64_t *ids, double *dists, int64_t *stats,
                     int32_t *flags)
{
    if (K < 1 || nprobe < 1 || nprobe > nc || delta_d < 1 || schedule < 0 || schedule > 3 ||
        ((schedule == 1 || schedule == 3) && tile < 1) || lag < 0 || seed < 0 ||
        (schedule == 3 && (lag > 0 || seed > 0)) || !(bias > -1.0))
        return -1;
    /* inverted lists, members in ascending id */
    int64_t *start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) start[assign[i] + 1] += 1;
    for (int c = 0; c < nc; ++c) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; ++i) members[start[assign[i]] + fill[assign[i]]++] = i;
    free(fill);
    double *Lam = prefix_lambda(lam, D);

    int32_t *probe = (int32_t *)malloc(sizeof(int32_t) * (size_t)nq * nprobe);
    int32_t *ptie = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nq > 0 ? nq : 1));
    or_probe(Qr, nq, D, cent, nc, nprobe, probe, ptie, tol);

    #pragma omp parallel
    {
        kv_t *buf = (kv_t *)malloc(sizeof(kv_t) * (size_t)(K + OR_PEND));
        double *hist = (double *)malloc(sizeof(double) * (size_t)(lag + 1));   /* r^2 after recent epochs */
        #pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const double *q = Qr + qi * D;
            const int32_t *pq = probe + qi * nprobe;
            int ntop = 0, npend = 0, tie = 0;
            int64_t epoch = 0;
            double dropped = INFINITY;   /* best squared distance accepted but not kept */
            int64_t st[4] = {0, 0, 0, 0};
            double r2_seed = INFINITY;
            /* one candidate against the epoch's threshold r2 (biased by the bracket) */
            #define OR_VISIT(id_, r2_)                                                               \
                do {                                                                                 \
                    double r2b = (r2_) * (1.0 + bias), d2 = 0.0;                                     \
                    int dims = 0;                                                                    \
                    int acc = dco(q, Xr + (id_) * D, D, delta_d, sqrt(r2b), r2b, Lam, eps,           \
                                  eps != NULL, tol, &d2, &dims, &tie);                               \
                    st[0] += 1;                                                                      \
                    st[1] += dims;                                                                   \
                    if (acc) {                                                                       \
                        st[2] += 1;                                                                  \
                        if (npend == OR_PEND) merge_pending(buf, &ntop, &npend, K, &dropped);        \
                        buf[ntop + npend].key = d2;                                                  \
                        buf[ntop + npend].id = (id_);                                                \
                        ++npend;                                                                     \
                    } else if (dims < D) st[3] += 1;                                                 \
                } while (0)
            if (schedule == 3) {
                int64_t lo = 0, hi = tile, longest = 0;
                for (int j = 0; j < nprobe; ++j)
                    if (start[pq[j] + 1] - start[pq[j]] > longest) longest = start[pq[j] + 1] - start[pq[j]];
                while (lo < longest) {
                    double r2 = ntop < K ? INFINITY : buf[K - 1].key;   /* after epochs 0..e-1 */
                    for (int j = 0; j < nprobe; ++j) {
                        int c = pq[j];
                        int64_t len = start[c + 1] - start[c];
                        for (int64_t t = lo; t < hi && t < len; ++t) OR_VISIT(members[start[c] + t], r2);
                    }
                    merge_pending(buf, &ntop, &npend, K, &dropped);
                    lo = hi;
                    hi = 2 * hi;
                }
            } else {
                for (int j = 0; j < nprobe; ++j) {
                    int c = pq[j];
                    if (seed > 0 && j == seed) r2_seed = ntop == K ? buf[K - 1].key : INFINITY;
                    int64_t len = start[c + 1] - start[c];
                    int64_t elen = schedule == 0 ? 1 : schedule == 1 ? tile : (len > 0 ? len : 1);
                    for (int64_t e0 = 0; e0 < len; e0 += elen) {
                        double r2 = ntop == K ? buf[K - 1].key : INFINITY;
                        if (lag > 0) r2 = epoch - 1 - lag >= 0 ? hist[(epoch - 1 - lag) % (lag + 1)] : INFINITY;
                        if (seed > 0 && j >= seed) r2 = r2_seed;
                        int64_t e1 = e0 + elen < len ? e0 + elen : len;
                        for (int64_t t = e0; t < e1; ++t) OR_VISIT(members[start[c] + t], r2);
                        merge_pending(buf, &ntop, &npend, K, &dropped);
                        if (lag > 0) hist[epoch % (lag + 1)] = ntop == K ? buf[K - 1].key : INFINITY;
                        ++epoch;
                    }
                }
            }
            #undef OR_VISIT
            if (ntop == K && isfinite(dropped) && near_tie(buf[K - 1].key, dropped, tol)) tie |= 4;
            for (int s = 0; s < K; ++s) {
                ids[qi * K + s] = s < ntop ? buf[s].id : -1;
                dists[qi * K + s] = s < ntop ? buf[s].key : INFINITY;
            }
            if (stats) for (int s = 0; s < 4; ++s) stats[qi * 4 + s] = st[s];
            if (flags) flags[qi] = tie | (ptie[qi] ? 8 : 0);
        }
        free(buf);
        free(hist);
    }
    free(probe); free(ptie); free(Lam); free(start); free(members);
    return 0;
}

/* Exact K nearest neighbours by brute force in FP64 (ground truth), ordered by
 * (squared distance, id).  X, Q are FP32 inputs in any common coordinates. */
OR_API void or_exact_knn(const float *X, int64_t n, int d, const float *Q, int64_t nq, int K,
                         int64_t *ids, double *dists)
{
    #pragma omp parallel
    {
        kv_t *buf = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
        #pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const float *q = Q + qi * d;
            for (int64_t i = 0; i < n; ++i) {
                const float *x = X + i * d;
                double s = 0.0;
                for (int k = 0; k < d; ++k) { double t = (double)q[k] - (double)x[k]; s += t * t; }
                buf[i].key = s;
                buf[i].id = i;
            }
            qsort(buf, (size_t)n, sizeof(kv_t), kv_cmp);
            for (int s = 0; s < K; ++s) {
                ids[qi * K + s] = s < n ? buf[s].id : -1;
                dists[qi * K + s] = s < n ? buf[s].key : INFINITY;
            }
        }
        free(buf);
    }
}

/* ------------------------------------------------------------------------ */
/* HNSW with DADE DCOs (HNSW*, Section 3.4; the graph of Section 4.1).       */
/* ------------------------------------------------------------------------ */

/* The (squared distance, id) order of every set below: 1 iff (ka, ia) < (kb, ib). */
static int kv_less(double ka, int64_t ia, double kb, int64_t ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

static double rel_gap(double a, double b)
{
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    return m > 0.0 ? fabs(a - b) / m : INFINITY;
}

/*
 * HNSW's neighbour selection heuristic (Malkov and Yashunin, "Efficient and
 * robust approximate nearest neighbor search using Hierarchical Navigable
 * Small World graphs", Algorithm 4, with neither candidate extension nor
 * kept pruned connections): the m candidates, ascending by (squared distance
 * to the node, id), are taken in order, and candidate e is kept iff it is
 * nearer to the node than to every candidate kept before it, until cap are
 * kept.  cand[i].key = squared distance of candidate i to the node.  Writes
 * the kept ids to out and returns how many; *gap is lowered to the relative
 * gap of every comparison made.
 */
static int select_heuristic(const double *Xr, int D, const kv_t *cand, int m, int cap, int64_t *out,
                            double *gap)
{
    int kept = 0;
    for (int i = 0; i < m && kept < cap; ++i) {
        const double *xe = Xr + cand[i].id * D;
        int keep = 1;
        for (int s = 0; s < kept; ++s) {
            double des = sqdist(xe, Xr + out[s] * D, D);
            double g = rel_gap(des, cand[i].key);
            if (g < *gap) *gap = g;
            if (!(cand[i].key < des)) { keep = 0; break; }
        }
        if (keep) out[kept++] = cand[i].id;
    }
    return kept;
}

/*
 * The layer-0 graph the beam search walks.  The paper takes HNSW's graph
 * from its reference library (M = 16, Section 4.1) and changes only the
 * DCOs of the search.  Reading: layer 0 built in one pass over exact
 * neighbours instead of by incremental insertion:
 *   1. C(u) = the kc nearest other objects of u, ascending by (squared
 *      distance, id);
 *   2. sel(u) = the heuristic over C(u), at most M kept;
 *   3. U(v) = sel(v) and every u with v in sel(u), distinct, ascending by
 *      (squared distance to v, id); the neighbours of v are U(v) when it
 *      holds at most M0, else the heuristic over U(v) with cap M0.
 * nbr: n x M0 ids in that order, unused slots -1.  gap_sel[u] (may be NULL):
 * the smallest relative gap among the decisions of steps 1-2 for u (the
 * kc-th / (kc+1)-th boundary, neighbouring candidates of C(u), every
 * heuristic comparison); gap_fin[v] (may be NULL) the same for step 3 when
 * the heuristic runs (neighbouring entries of U(v), its comparisons).
 * Returns 0, or -1 on bad arguments.
 */
OR_API int or_hnsw_graph(const double *Xr, int64_t n, int D, int kc, int M, int M0, int32_t *nbr,
                         double *gap_sel, double *gap_fin)
{
    if (n < 1 || kc < 1 || M < 1 || M0 < 1) return -1;
    int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * M);
    int *nsel = (int *)malloc(sizeof(int) * (size_t)n);
    #pragma omp parallel
    {
        kv_t *buf = (kv_t *)malloc(sizeof(kv_t) * (size_t)n);
        #pragma omp for schedule(dynamic, 16)
        for (int64_t u = 0; u < n; ++u) {
            int64_t m = 0;
            for (int64_t i = 0; i < n; ++i) {
                if (i == u) continue;
                buf[m].key = sqdist(Xr + u * D, Xr + i * D, D);
                buf[m].id = i;
                ++m;
            }
            qsort(buf, (size_t)m, sizeof(kv_t), kv_cmp);
            int kk = (int)(m < kc ? m : kc);
            double g = INFINITY;
            if (kk < m) g = rel_gap(buf[kk - 1].key, buf[kk].key);
            for (int i = 0; i + 1 < kk; ++i) {
                double gi = rel_gap(buf[i].key, buf[i + 1].key);
                if (gi < g) g = gi;
            }
            nsel[u] = select_heuristic(Xr, D, buf, kk, M, sel + u * M, &g);
            if (gap_sel) gap_sel[u] = g;
        }
        free(buf);
    }
    /* reverse entries: u joins U(v) for every v in sel(u) */
    int64_t *rstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t u = 0; u < n; ++u)
        for (int s = 0; s < nsel[u]; ++s) rstart[sel[u * M + s] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) rstart[v + 1] += rstart[v];
    int64_t *rev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rstart[n] > 0 ? rstart[n] : 1));
    int64_t *rfill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    for (int64_t u = 0; u < n; ++u)
        for (int s = 0; s < nsel[u]; ++s) {
            int64_t v = sel[u * M + s];
            rev[rstart[v] + rfill[v]++] = u;
        }
    free(rfill);
    #pragma omp parallel
    {
        int64_t cap = M;
        for (int64_t v = 0; v < n; ++v)
            if (rstart[v + 1] - rstart[v] + M > cap) cap = rstart[v + 1] - rstart[v] + M;
        kv_t *U = (kv_t *)malloc(sizeof(kv_t) * (size_t)cap);
        int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)M0);
        #pragma omp for schedule(dynamic, 16)
        for (int64_t v = 0; v < n; ++v) {
            int64_t m = 0;
            for (int s = 0; s < nsel[v]; ++s) {
                U[m].id = sel[v * M + s];
                U[m].key = sqdist(Xr + v * D, Xr + U[m].id * D, D);
                ++m;
            }
            for (int64_t t = rstart[v]; t < rstart[v + 1]; ++t) {
                U[m].id = rev[t];
                U[m].key = sqdist(Xr + v * D, Xr + rev[t] * D, D);
                ++m;
            }
            qsort(U, (size_t)m, sizeof(kv_t), kv_cmp);
            int64_t w = 0;   /* distinct ids: an id met twice has the same key, so the copies are adjacent */
            for (int64_t i = 0; i < m; ++i)
                if (w == 0 || U[i].id != U[w - 1].id) U[w++] = U[i];
            m = w;
            double g = INFINITY;
            int nk;
            if (m <= M0) {
                nk = (int)m;
                for (int64_t i = 0; i < m; ++i) kept[i] = U[i].id;
            } else {
                for (int64_t i = 0; i + 1 < m; ++i) {
                    double gi = rel_gap(U[i].key, U[i + 1].key);
                    if (gi < g) g = gi;
                }
                nk = select_heuristic(Xr, D, U, (int)m, M0, kept, &g);
            }
            for (int s = 0; s < M0; ++s) nbr[v * M0 + s] = s < nk ? (int32_t)kept[s] : -1;
            if (gap_fin) gap_fin[v] = g;
        }
        free(U);
        free(kept);
    }
    free(sel); free(nsel); free(rstart); free(rev);
    return 0;
}

/* R holds *nR objects ascending by (key, id), at most ef: put x in, dropping
 * the farthest when it would hold ef + 1.  Flag 8 when the dropped object and
 * the new farthest are within tol. */
static void r_insert(kv_t *R, int *nR, int ef, kv_t x, double tol, int *tie)
{
    int p = *nR;
    while (p > 0 && kv_less(x.key, x.id, R[p - 1].key, R[p - 1].id)) --p;
    if (*nR == ef) {
        if (p == ef) {
            if (near_tie(x.key, R[ef - 1].key, tol)) *tie |= 8;
            return;
        }
        double dropped = R[ef - 1].key;
        memmove(R + p + 1, R + p, sizeof(kv_t) * (size_t)(ef - 1 - p));
        R[p] = x;
        if (near_tie(dropped, R[ef - 1].key, tol)) *tie |= 8;
        return;
    }
    memmove(R + p + 1, R + p, sizeof(kv_t) * (size_t)(*nR - p));
    R[p] = x;
    *nR += 1;
}

/*
 * Algorithm 1 in the arithmetic of the paper's implementation (scalar FP32
 * C++, Section 4.1): t = q_k - o_k, t * t and the running sum each rounded to
 * FP32, dimensions in order (this file is built with contraction off, so no
 * fused multiply-add merges the steps).  The test of Section 3.3 in its
 * squared form, P_d > c_j r^2 with c_j = (1 + eps_d)^2 Lambda_d / Lambda_D
 * given in FP32 (coef[j] for the j-th tested d) and the product rounded to
 * FP32; at d = D accept iff P_D <= r^2.  coef == NULL: FDScanning.  The
 * result and tie bits as dco().
 */
static int dco_f32(const float *q, const float *o, int D, int delta_d, float r2, const float *coef, double tol,
                   float *dist2, int *dims, int *tie)
{
    int d = 0, j = 0;
    float P = 0.0f;
    while (d < D) {
        int dn = d + delta_d;
        if (dn > D) dn = D;
        for (int k = d; k < dn; ++k) {
            float t = q[k] - o[k];
            float sq = t * t;
            P = P + sq;
        }
        d = dn;
        if (d < D) {
            if (coef) {
                float bound = coef[j] * r2;
                if (isfinite(r2) && near_tie(P, bound, tol)) *tie |= 1;
                if (P > bound) { *dims = d; return 0; }
            }
            ++j;
        } else {
            if (isfinite(r2) && near_tie(P, r2, tol)) *tie |= 2;
            break;
        }
    }
    *dims = D;
    *dist2 = P;
    return P <= r2;
}

/*
 * Greedy beam search on the layer-0 graph with one DCO per neighbour
 * (Section 3.4): a search set S, unbounded, and a result set R of at most ef
 * objects, both ordered by (squared distance, id).  First every entry object
 * is visited with r = +inf (its exact distance) and enters S and R.  Then:
 *   stop when the visit budget is spent (max_visits > 0 and max_visits DCOs
 *       run) or S is empty;
 *   pop c, the nearest object of S; stop when c is farther than the farthest
 *       object of R (the search-layer stop of Malkov and Yashunin, Algorithm 2);
 *   for each neighbour e of c, in slot order, not yet visited: mark e visited
 *       and run the DCO (Algorithm 1) against r = the farthest distance in R
 *       (+inf while R holds fewer than ef); on accept e enters S and R, and R
 *       drops its farthest object when it would hold ef + 1.
 * schedule 0 (SEQUENTIAL): r is read before every DCO, the paper's order.
 * schedule 1 (NODE): r is read once when c is popped and serves all of c's
 *   neighbours; the accepted ones then enter S and R together (R keeps the
 *   ef nearest of R and them).  A stale r only accepts more.
 * The entry objects form one such group against r = +inf in both schedules.
 * Arithmetic: with Xr, Qr (FP64) the DCOs are dco() with eps (NULL:
 * FDScanning) and bias as or_search; with Xr32, Qr32 (FP32, Xr and Qr NULL)
 * they are dco_f32() with coef32 (NULL: FDScanning), every distance an FP32
 * value, bias unused.
 * Results: the K nearest of R by (squared distance, id); missing slots
 * (-1, +inf).  entry: nq x n_entry object ids (negative or out-of-range slots
 * skipped); nbr: n x M0 ids (-1 unused).
 * stats (nq x 5, may be NULL): DCOs run, sum of dims used, accepted, pruned,
 * objects popped and expanded.
 * flags (nq, may be NULL): 1|2 DCO near-ties (see dco); 4 a near-tie in the
 * pop order (another object of S within tol of the popped one) or in the stop
 * compare; 8 a near-tie at an eviction from R; 16 the K-th and (K+1)-th of R
 * within tol at the end; 32 the visit budget ended the search.
 * Returns 0, or -1 on bad arguments.
 */
OR_API int or_hnsw_search(const double *Xr, const float *Xr32, int64_t n, int D, const int32_t *nbr, int M0,
                          const double *lam, const double *Qr, const float *Qr32, int64_t nq, const int64_t *entry,
                          int n_entry, int K, int ef, int delta_d, const double *eps, const float *coef32,
                          int schedule, int64_t max_visits, double tol, double bias, int64_t *ids, double *dists,
                          int64_t *stats, int32_t *flags)
{
    const int f32 = Xr32 != NULL;
    if (n < 1 || K < 1 || ef < K || M0 < 1 || n_entry < 1 || delta_d < 1 || schedule < 0 || schedule > 1 ||
        !(bias > -1.0) || (f32 ? (Qr32 == NULL || Xr != NULL || Qr != NULL) : (Xr == NULL || Qr == NULL)))
        return -1;
    double *Lam = prefix_lambda(lam, D);
    #pragma omp parallel
    {
        unsigned char *vis = (unsigned char *)calloc((size_t)n, 1);
        int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        kv_t *R = (kv_t *)malloc(sizeof(kv_t) * (size_t)(ef + M0 + n_entry + 1));
        kv_t *S = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n + 1));
        kv_t *acc = (kv_t *)malloc(sizeof(kv_t) * (size_t)(M0 + n_entry));
        #pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; ++qi) {
            int nR = 0, nS = 0, tie = 0, na = 0;
            int64_t nt = 0, st[5] = {0, 0, 0, 0, 0};
            /* one DCO of object e_ against the squared threshold r2_ */
            #define OR_HVISIT(e_, r2_)                                                                  \
                do {                                                                                    \
                    int dims = 0, ok;                                                                   \
                    double d2 = 0.0;                                                                    \
                    vis[e_] = 1;                                                                        \
                    touched[nt++] = (e_);                                                               \
                    if (f32) {                                                                          \
                        float p32 = 0.0f;                                                               \
                        ok = dco_f32(Qr32 + qi * D, Xr32 + (e_) * D, D, delta_d, (float)(r2_), coef32,  \
                                     tol, &p32, &dims, &tie);                                           \
                        d2 = p32;                                                                       \
                    } else {                                                                            \
                        double r2b = (r2_) * (1.0 + bias);                                              \
                        ok = dco(Qr + qi * D, Xr + (e_) * D, D, delta_d, sqrt(r2b), r2b, Lam, eps,      \
                                 eps != NULL, tol, &d2, &dims, &tie);                                   \
                    }                                                                                   \
                    st[0] += 1;                                                                         \
                    st[1] += dims;                                                                      \
                    if (ok) {                                                                           \
                        st[2] += 1;                                                                     \
                        acc[na].key = d2;                                                               \
                        acc[na].id = (e_);                                                              \
                        ++na;                                                                           \
                    } else if (dims < D) st[3] += 1;                                                    \
                } while (0)
            /* the accepted group enters S and R together: R keeps the ef nearest */
            #define OR_HADMIT()                                                                         \
                do {                                                                                    \
                    for (int a_ = 0; a_ < na; ++a_) S[nS++] = acc[a_];                                  \
                    if (na > 0) {                                                                       \
                        memcpy(R + nR, acc, sizeof(kv_t) * (size_t)na);                                 \
                        qsort(R, (size_t)(nR + na), sizeof(kv_t), kv_cmp);                              \
                        nR += na;                                                                       \
                        if (nR > ef) {                                                                  \
                            if (near_tie(R[ef - 1].key, R[ef].key, tol)) tie |= 8;                      \
                            nR = ef;                                                                    \
                        }                                                                               \
                    }                                                                                   \
                    na = 0;                                                                             \
                } while (0)
            for (int j = 0; j < n_entry; ++j) {
                int64_t e = entry[qi * n_entry + j];
                if (e < 0 || e >= n || vis[e]) continue;
                OR_HVISIT(e, INFINITY);
            }
            OR_HADMIT();
            for (;;) {
                if (max_visits > 0 && st[0] >= max_visits) { tie |= 32; break; }
                if (nS == 0) break;
                int b = 0;
                for (int i = 1; i < nS; ++i)
                    if (kv_less(S[i].key, S[i].id, S[b].key, S[b].id)) b = i;
                kv_t c = S[b];
                for (int i = 0; i < nS; ++i)
                    if (i != b && near_tie(S[i].key, c.key, tol)) { tie |= 4; break; }
                S[b] = S[--nS];
                const kv_t far = R[nR - 1];
                if (far.id != c.id && near_tie(c.key, far.key, tol)) tie |= 4;
                if (kv_less(far.key, far.id, c.key, c.id)) break;
                st[4] += 1;
                const double r2_node = nR == ef ? R[ef - 1].key : INFINITY;
                for (int s = 0; s < M0; ++s) {
                    int64_t e = nbr[c.id * M0 + s];
                    if (e < 0 || e >= n || vis[e]) continue;
                    if (schedule == 0) {
                        OR_HVISIT(e, nR == ef ? R[ef - 1].key : INFINITY);
                        if (na > 0) {
                            S[nS++] = acc[0];
                            r_insert(R, &nR, ef, acc[0], tol, &tie);
                            na = 0;
                        }
                    } else {
                        OR_HVISIT(e, r2_node);
                    }
                }
                if (schedule == 1) OR_HADMIT();
            }
            #undef OR_HVISIT
            #undef OR_HADMIT
            if (nR > K && near_tie(R[K - 1].key, R[K].key, tol)) tie |= 16;
            for (int s = 0; s < K; ++s) {
                ids[qi * K + s] = s < nR ? R[s].id : -1;
                dists[qi * K + s] = s < nR ? R[s].key : INFINITY;
            }
            if (stats) for (int s = 0; s < 5; ++s) stats[qi * 5 + s] = st[s];
            if (flags) flags[qi] = tie;
            for (int64_t t = 0; t < nt; ++t) vis[touched[t]] = 0;
        }
        free(vis); free(touched); free(R); free(S); free(acc);
    }
    free(Lam);
    return 0;
}
