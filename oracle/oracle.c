/*
 * CPU FP64 oracle for the batched one-dimensional complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the CPU baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the GPU library, and the library never
 * calls it: the product path has no CPU fallback.
 *
 * Data layout: `x` and `y` hold `batch` rows of `n` complex values each, row i
 * starting at complex element i*n, every complex value stored as two doubles
 * (re, im).  `sign` is the sign of the exponent: -1 is the forward transform
 * (omega_N = exp(-2*pi*i/N), Sec. II), +1 the unnormalised inverse.
 *
 * Three transforms, all in FP64:
 *
 *   oracle_dft_naive   - the DFT definition of Sec. II written out: the dense
 *                        product DFT_N * x with DFT_N[m][k] = omega_N^(m*k),
 *                        accumulated term by term in index order.
 *   oracle_fft_radix2  - the textbook recursive radix-2 decimation-in-time FFT
 *                        (Cooley-Tukey, Sec. II), for power-of-two n.
 *   oracle_fft_eq2     - the general-radix recursion of Eq. 2,
 *                        DFT_N = (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K,
 *                        applied right to left with K the smallest prime factor
 *                        of N and recursing on DFT_M.  The paper leaves the
 *                        entries of D^N_M and Pi^N_K to its 4-point example
 *                        (Eq. 1); the readings used are
 *                          (Pi^N_K x)[k*M + m] = x[m*K + k]
 *                          D^N_M = diag(omega_N^(k*j)) at position k*M + j,
 *                        both of which reproduce Eq. 1 at N = 4.
 *
 * Every root of unity omega_N^e is evaluated as cos/sin of 2*pi*(e mod N)/N
 * with the exponent reduced exactly in integers first.
 *
 * Return codes: 0 success, -1 invalid argument, -2 out of memory.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static const double kTwoPi = 6.28318530717958647692528676655900577;

/* omega_N^e for the transform direction `sign`: exp(sign * 2*pi*i * e / N). */
static void root_of_unity(int64_t N, int64_t e, int sign, double *re, double *im) {
    int64_t r = e % N;
    if (r < 0) r += N;
    double angle = kTwoPi * (double)r / (double)N;
    *re = cos(angle);
    *im = (double)sign * sin(angle);
}

/* ------------------------------------------------------------------------ */
/* Direct DFT: y[m] = sum_k omega_N^(m*k) x[k]   (Sec. II, DFT_N definition) */
/* ------------------------------------------------------------------------ */

/* The N roots omega_N^j, j < N, so that DFT_N[m][k] is table[(m*k) mod N]. */
static double *roots_table(int64_t N, int sign) {
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!t) return NULL;
    for (int64_t j = 0; j < N; ++j) root_of_unity(N, j, sign, &t[2 * j], &t[2 * j + 1]);
    return t;
}

static void dft_row(const double *x, double *y, int64_t N, const double *roots) {
    for (int64_t m = 0; m < N; ++m) {
        double acc_re = 0.0, acc_im = 0.0;
        for (int64_t k = 0; k < N; ++k) {
            int64_t e = (m * k) % N;
            double wr = roots[2 * e], wi = roots[2 * e + 1];
            double xr = x[2 * k], xi = x[2 * k + 1];
            acc_re += wr * xr - wi * xi;
            acc_im += wr * xi + wi * xr;
        }
        y[2 * m] = acc_re;
        y[2 * m + 1] = acc_im;
    }
}

/* ------------------------------------------------------------------------ */
/* Recursive radix-2 decimation in time (Cooley-Tukey, Sec. II).             */
/* X[k] = E[k] + omega_N^k O[k],  X[k + N/2] = E[k] - omega_N^k O[k], where   */
/* E and O are the half-length DFTs of the even and odd samples.             */
/* ------------------------------------------------------------------------ */

static void radix2_rec(const double *x, int64_t stride, double *y, int64_t N, int sign) {
    if (N == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    int64_t h = N / 2;
    radix2_rec(x, 2 * stride, y, h, sign);                /* even samples -> y[0, h)  */
    radix2_rec(x + 2 * stride, 2 * stride, y + 2 * h, h, sign); /* odd samples -> y[h, N) */
    for (int64_t k = 0; k < h; ++k) {
        double wr, wi;
        root_of_unity(N, k, sign, &wr, &wi);
        double er = y[2 * k], ei = y[2 * k + 1];
        double or_ = y[2 * (k + h)], oi = y[2 * (k + h) + 1];
        double tr = wr * or_ - wi * oi;
        double ti = wr * oi + wi * or_;
        y[2 * k] = er + tr;
        y[2 * k + 1] = ei + ti;
        y[2 * (k + h)] = er - tr;
        y[2 * (k + h) + 1] = ei - ti;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: DFT_N = (DFT_K (x) I_M) . D^N_M . (I_K (x) DFT_M) . Pi^N_K,  N = MK */
/* ------------------------------------------------------------------------ */

static int64_t smallest_prime_factor(int64_t N) {
    for (int64_t p = 2; p * p <= N; ++p)
        if (N % p == 0) return p;
    return N;
}

static int eq2_rec(const double *x, double *y, int64_t N, int sign) {
    if (N == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return ORACLE_OK;
    }
    int64_t K = smallest_prime_factor(N);
    if (K == N) { /* prime length: the direct DFT of Sec. II */
        double *roots = roots_table(N, sign);
        if (!roots) return ORACLE_ENOMEM;
        dft_row(x, y, N, roots);
        free(roots);
        return ORACLE_OK;
    }
    int64_t M = N / K;
    double *v = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *z = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!v || !z) {
        free(v);
        free(z);
        return ORACLE_ENOMEM;
    }
    /* Pi^N_K: gather at stride K, so block k holds x[k], x[k+K], x[k+2K], ... */
    for (int64_t k = 0; k < K; ++k)
        for (int64_t m = 0; m < M; ++m) {
            v[2 * (k * M + m)] = x[2 * (m * K + k)];
            v[2 * (k * M + m) + 1] = x[2 * (m * K + k) + 1];
        }
    /* I_K (x) DFT_M: a length-M DFT of each of the K contiguous blocks. */
    for (int64_t k = 0; k < K; ++k) {
        int rc = eq2_rec(v + 2 * k * M, z + 2 * k * M, M, sign);
        if (rc != ORACLE_OK) {
            free(v);
            free(z);
            return rc;
        }
    }
    /* D^N_M: entry k*M + j is scaled by omega_N^(k*j). */
    for (int64_t k = 0; k < K; ++k)
        for (int64_t j = 0; j < M; ++j) {
            double wr, wi;
            root_of_unity(N, k * j, sign, &wr, &wi);
            double zr = z[2 * (k * M + j)], zi = z[2 * (k * M + j) + 1];
            z[2 * (k * M + j)] = wr * zr - wi * zi;
            z[2 * (k * M + j) + 1] = wr * zi + wi * zr;
        }
    /* DFT_K (x) I_M: a length-K DFT across the blocks, at stride M. */
    for (int64_t j2 = 0; j2 < K; ++j2)
        for (int64_t j1 = 0; j1 < M; ++j1) {
            double acc_re = 0.0, acc_im = 0.0;
            for (int64_t k = 0; k < K; ++k) {
                double wr, wi;
                root_of_unity(K, j2 * k, sign, &wr, &wi);
                double zr = z[2 * (k * M + j1)], zi = z[2 * (k * M + j1) + 1];
                acc_re += wr * zr - wi * zi;
                acc_im += wr * zi + wi * zr;
            }
            y[2 * (j2 * M + j1)] = acc_re;
            y[2 * (j2 * M + j1) + 1] = acc_im;
        }
    free(v);
    free(z);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Batch driver: rows are independent; a static split of rows over threads. */
/* ------------------------------------------------------------------------ */

enum { KIND_NAIVE = 0, KIND_RADIX2 = 1, KIND_EQ2 = 2 };

typedef struct {
    const double *x;
    double *y;
    int64_t n, row_begin, row_end;
    int sign, kind, status;
} job_t;

static void *run_rows(void *arg) {
    job_t *j = (job_t *)arg;
    double *roots = NULL;
    if (j->kind == KIND_NAIVE) {
        roots = roots_table(j->n, j->sign);
        if (!roots) {
            j->status = ORACLE_ENOMEM;
            return NULL;
        }
    }
    for (int64_t r = j->row_begin; r < j->row_end; ++r) {
        const double *xr = j->x + 2 * r * j->n;
        double *yr = j->y + 2 * r * j->n;
        if (j->kind == KIND_NAIVE) {
            dft_row(xr, yr, j->n, roots);
        } else if (j->kind == KIND_RADIX2) {
            radix2_rec(xr, 1, yr, j->n, j->sign);
        } else {
            int rc = eq2_rec(xr, yr, j->n, j->sign);
            if (rc != ORACLE_OK) {
                j->status = rc;
                break;
            }
        }
    }
    free(roots);
    return NULL;
}

static int run_batch(const double *x, double *y, int64_t n, int64_t batch, int sign,
                     int nthreads, int kind) {
    if (!x || !y || n < 1 || batch < 0 || (sign != -1 && sign != 1)) return ORACLE_EINVAL;
    if (kind == KIND_RADIX2 && (n & (n - 1)) != 0) return ORACLE_EINVAL;
    if (x == y) return ORACLE_EINVAL; /* out of place only */
    if (batch == 0) return ORACLE_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > batch) nthreads = (int)batch;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return ORACLE_ENOMEM;
    }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].x = x;
        jobs[t].y = y;
        jobs[t].n = n;
        jobs[t].row_begin = batch * t / nthreads;
        jobs[t].row_end = batch * (t + 1) / nthreads;
        jobs[t].sign = sign;
        jobs[t].kind = kind;
        jobs[t].status = ORACLE_OK;
    }
    int status = ORACLE_OK;
    if (nthreads == 1) {
        run_rows(&jobs[0]);
    } else {
        int started = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (pthread_create(&tids[t], NULL, run_rows, &jobs[t]) != 0) break;
            ++started;
        }
        for (int t = started; t < nthreads; ++t) run_rows(&jobs[t]); /* inline leftovers */
        for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    }
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status != ORACLE_OK) status = jobs[t].status;
    free(jobs);
    free(tids);
    return status;
}

int oracle_dft_naive(const double *x, double *y, int64_t n, int64_t batch, int sign, int nthreads) {
    return run_batch(x, y, n, batch, sign, nthreads, KIND_NAIVE);
}

int oracle_fft_radix2(const double *x, double *y, int64_t n, int64_t batch, int sign, int nthreads) {
    return run_batch(x, y, n, batch, sign, nthreads, KIND_RADIX2);
}

int oracle_fft_eq2(const double *x, double *y, int64_t n, int64_t batch, int sign, int nthreads) {
    return run_batch(x, y, n, batch, sign, nthreads, KIND_EQ2);
}
