/*
 * FP64 CPU oracle for the batched complex FFT -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline /
 * reference leg may load this library.  The product path (the CUDA library and
 * its Python binding) never links, imports or calls it, and shares no code
 * with it.
 *
 * What it computes (Bergach et al., "Efficient FFT mapping on GPU for radar
 * processing application", Sec. 2.1, the DFT equation):
 *
 *     X(k) = sum_{n=0}^{N-1} x(n) * w_N^{n k},   w_N = exp(-2 pi i / N)
 *
 * and the backward transform obtained by flipping the sign of the exponent
 * (same section).  The paper does not state a normalisation for the backward
 * transform; this oracle reads it as unnormalised, so backward(forward(x)) = N x.
 *
 * Two routes to the same numbers:
 *   oracle_dft  -- the definition written out, O(N^2), for small N;
 *   oracle_fft  -- textbook recursive radix-2 decimation in time
 *                  (Cooley & Tukey 1965): the DFT reached exactly up to
 *                  rounding, O(N log N), used for large N.
 * 2D transforms are 1D transforms along rows, then along columns
 * (separability of the 2D DFT).
 *
 * Data: complex values are interleaved (re, im) doubles.  Batched 1D element
 * (b, i) is at b*n + i; a 2D frame is row-major [rows][cols], batch-major.
 * sign = -1 forward, +1 backward.  Functions return 0 on success, -1 on a bad
 * argument.  `threads` <= 0 means "all online cores"; the batch (or the set of
 * rows / columns) is split over POSIX threads, each transform is sequential.
 *
 * Compile with -ffp-contract=off so x86 and Arm hosts round identically.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct { double re, im; } cd;

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/*
 * w_n^m = exp(sign * 2 pi i m / n) in FP64.  The integer exponent is reduced
 * mod n exactly, then the angle theta = 2 pi m / n is folded into [0, pi/4]
 * by up to three reflections done on the integer m (so they are exact; the
 * second needs n even and the third n divisible by 4, otherwise the angle
 * is used as it stands):
 *   theta > pi   :  theta -> 2pi - theta   (cos same, sin negated)
 *   theta > pi/2 :  theta -> pi - theta    (cos negated, sin same)
 *   theta > pi/4 :  theta -> pi/2 - theta  (cos and sin swapped)
 * Multiples of pi/2 therefore come out exact and the table is symmetric.
 */
static cd unit_root(int64_t m, int64_t n, int sign) {
    m %= n;
    if (m < 0) m += n;
    int neg_s = 0, neg_c = 0, swap = 0;
    if (2 * m > n) { m = n - m; neg_s = 1; }
    if (n % 2 == 0 && 4 * m > n) { m = n / 2 - m; neg_c = 1; }
    if (n % 4 == 0 && 8 * m > n) { m = n / 4 - m; swap = 1; }
    double th = 2.0 * M_PI * (double)m / (double)n;
    double c = cos(th), s = sin(th);
    if (swap) { double t = c; c = s; s = t; }
    if (neg_c) c = -c;
    if (neg_s) s = -s;
    cd w;
    w.re = c;
    w.im = (double)sign * s;
    return w;
}

/* ------------------------------------------------------------------ DFT -- */

/* Direct evaluation of the DFT definition, O(n^2).  The exponent n*k is
 * reduced mod n as an integer before the root is evaluated. */
int oracle_dft(const double *x, double *X, int64_t n, int sign) {
    if (!x || !X || n < 1 || (sign != 1 && sign != -1)) return -1;
    const cd *xi = (const cd *)x;
    cd *Xo = (cd *)malloc(sizeof(cd) * (size_t)n);
    if (!Xo) return -1;
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            cd w = unit_root((j * k) % n, n, sign);
            sr += xi[j].re * w.re - xi[j].im * w.im;
            si += xi[j].re * w.im + xi[j].im * w.re;
        }
        Xo[k].re = sr;
        Xo[k].im = si;
    }
    memcpy(X, Xo, sizeof(cd) * (size_t)n);
    free(Xo);
    return 0;
}

/* ------------------------------------------------- recursive radix-2 FFT -- */

/* Radix-2 decimation in time: X = E + w^k O over the even- and odd-indexed
 * halves.  `w` holds w_N^j for j < N/2 of the top-level length N; a
 * sub-transform of length len uses w_len^k = w_N^{k * (N/len)}. */
static void fft_rec(const cd *x, int64_t xstride, cd *X, int64_t len,
                    const cd *w, int64_t wstride) {
    if (len == 1) { X[0] = x[0]; return; }
    int64_t h = len / 2;
    fft_rec(x, 2 * xstride, X, h, w, 2 * wstride);
    fft_rec(x + xstride, 2 * xstride, X + h, h, w, 2 * wstride);
    for (int64_t k = 0; k < h; ++k) {
        cd e = X[k], o = X[k + h], t;
        cd wk = w[k * wstride];
        t.re = wk.re * o.re - wk.im * o.im;
        t.im = wk.re * o.im + wk.im * o.re;
        X[k].re = e.re + t.re;     X[k].im = e.im + t.im;
        X[k + h].re = e.re - t.re; X[k + h].im = e.im - t.im;
    }
}

static cd *make_table(int64_t n, int sign) {
    int64_t h = n / 2 > 0 ? n / 2 : 1;
    cd *w = (cd *)malloc(sizeof(cd) * (size_t)h);
    if (!w) return NULL;
    for (int64_t j = 0; j < h; ++j) w[j] = unit_root(j, n, sign);
    return w;
}

/* One transform, strided input and output (strides in complex elements). */
static void fft_one(const cd *x, int64_t xs, cd *X, int64_t xo, int64_t n,
                    const cd *w, cd *tmp_in, cd *tmp_out) {
    for (int64_t i = 0; i < n; ++i) tmp_in[i] = x[i * xs];
    fft_rec(tmp_in, 1, tmp_out, n, w, 1);
    for (int64_t i = 0; i < n; ++i) X[i * xo] = tmp_out[i];
}

typedef struct {
    const cd *x; cd *X;
    int64_t n, count;          /* transform length, number of transforms */
    int64_t in_elem, in_tr;    /* strides: between elements, between transforms */
    int64_t out_elem, out_tr;
    const cd *w;
    int64_t begin, end;
    int err;
} job_t;

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    cd *a = (cd *)malloc(sizeof(cd) * (size_t)j->n);
    cd *b = (cd *)malloc(sizeof(cd) * (size_t)j->n);
    if (!a || !b) { j->err = 1; free(a); free(b); return NULL; }
    for (int64_t t = j->begin; t < j->end; ++t)
        fft_one(j->x + t * j->in_tr, j->in_elem, j->X + t * j->out_tr,
                j->out_elem, j->n, j->w, a, b);
    free(a); free(b);
    return NULL;
}

static int resolve_threads(int threads) {
    if (threads > 0) return threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* `count` transforms of length n with the given strides, split over threads. */
static int run_many(const cd *x, cd *X, int64_t n, int64_t count,
                    int64_t in_elem, int64_t in_tr, int64_t out_elem,
                    int64_t out_tr, int sign, int threads) {
    if (count == 0) return 0;
    cd *w = make_table(n, sign);
    if (!w) return -1;
    int nt = resolve_threads(threads);
    if ((int64_t)nt > count) nt = (int)count;
    job_t *jobs = (job_t *)calloc((size_t)nt, sizeof(job_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    if (!jobs || !tid) { free(w); free(jobs); free(tid); return -1; }
    int rc = 0;
    for (int i = 0; i < nt; ++i) {
        job_t *j = &jobs[i];
        j->x = x; j->X = X; j->n = n; j->count = count;
        j->in_elem = in_elem; j->in_tr = in_tr;
        j->out_elem = out_elem; j->out_tr = out_tr; j->w = w;
        j->begin = count * i / nt; j->end = count * (i + 1) / nt;
    }
    char *started = (char *)calloc((size_t)nt, 1);
    if (!started) { free(w); free(jobs); free(tid); return -1; }
    for (int i = 1; i < nt; ++i)
        started[i] = pthread_create(&tid[i], NULL, worker, &jobs[i]) == 0;
    worker(&jobs[0]);                          /* this thread takes part 0 */
    for (int i = 1; i < nt; ++i) {
        if (started[i]) pthread_join(tid[i], NULL);
        else worker(&jobs[i]);                 /* no thread: run it here */
    }
    free(started);
    for (int i = 0; i < nt; ++i) if (jobs[i].err) rc = -1;
    free(w); free(jobs); free(tid);
    return rc;
}

/* Batched 1D FFT: x, X hold batch*n interleaved complex doubles. */
int oracle_fft(const double *x, double *X, int64_t n, int64_t batch, int sign,
               int threads) {
    if (!x || !X || !is_pow2(n) || batch < 0 || (sign != 1 && sign != -1))
        return -1;
    return run_many((const cd *)x, (cd *)X, n, batch, 1, n, 1, n, sign, threads);
}

/* Batched 2D FFT of row-major [rows][cols] frames: rows first, then columns. */
int oracle_fft2d(const double *x, double *X, int64_t rows, int64_t cols,
                 int64_t batch, int sign, int threads) {
    if (!x || !X || !is_pow2(rows) || !is_pow2(cols) || batch < 0 ||
        (sign != 1 && sign != -1))
        return -1;
    const cd *xi = (const cd *)x;
    cd *Xo = (cd *)X;
    for (int64_t b = 0; b < batch; ++b) {
        const cd *src = xi + b * rows * cols;
        cd *dst = Xo + b * rows * cols;
        /* along each row: contiguous elements, rows at distance cols */
        if (run_many(src, dst, cols, rows, 1, cols, 1, cols, sign, threads))
            return -1;
        /* along each column: elements at distance cols, columns adjacent;
         * computed in place on dst (each column is gathered first) */
        if (run_many(dst, dst, rows, cols, cols, 1, cols, 1, sign, threads))
            return -1;
    }
    return 0;
}

/* Samples a subset of transforms of a batched 1D problem: transform
 * indices idx[0..m) of the batch held in x (batch*n values). */
int oracle_fft_select(const double *x, double *X, int64_t n, const int64_t *idx,
                      int64_t m, int sign, int threads) {
    if (!x || !X || !idx || !is_pow2(n) || m < 0 || (sign != 1 && sign != -1))
        return -1;
    cd *w = make_table(n, sign);
    if (!w) return -1;
    cd *a = (cd *)malloc(sizeof(cd) * (size_t)n);
    cd *b = (cd *)malloc(sizeof(cd) * (size_t)n);
    if (!a || !b) { free(w); free(a); free(b); return -1; }
    (void)threads;                 /* samples are few: sequential */
    for (int64_t t = 0; t < m; ++t)
        fft_one((const cd *)x + idx[t] * n, 1, (cd *)X + t * n, 1, n, w, a, b);
    free(w); free(a); free(b);
    return 0;
}

/* The FP64 root of unity itself, for pinning the table. */
int oracle_unit_root(int64_t m, int64_t n, int sign, double *out2) {
    if (!out2 || n < 1 || (sign != 1 && sign != -1)) return -1;
    cd w = unit_root(m, n, sign);
    out2[0] = w.re; out2[1] = w.im;
    return 0;
}

int oracle_num_threads(int threads) { return resolve_threads(threads); }
