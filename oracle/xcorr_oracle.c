/*
 * X-stage oracle: a plain CPU cross-multiply-and-integrate.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this file's library; the CUDA library
 * shares no code, header, table or helper with it.
 *
 * What it computes (Sec. 1: the X-stage is an outer product of the per-antenna
 * spectra for one time and frequency; Sec. 2.1: cross multiplication and
 * integration of the products for each frequency channel and time sample;
 * Sec. 2.2.3, Eq. 1: all N_i (N_i + 1) / 2 input pairs, autos included), for
 * every channel c and every input pair j <= i:
 *
 *     V[c][i][j] = sum_{t < K} x[t][c][i] * conj(x[t][c][j])
 *     Re = sum (xr_i xr_j + xi_i xi_j),  Im = sum (xi_i xr_j - xr_i xi_j)
 *
 * Input i is (station i / 2, polarisation i % 2), following the sample order
 * [time][channel][station][pol].  The output is the packed lower triangle,
 * pair index i (i + 1) / 2 + j, with (re, im) interleaved, [channel][pair][2].
 * Integer inputs accumulate in int64 and float inputs in double; the result is
 * the integrated SUM over the K samples (the paper's GPU averages; the sum
 * keeps the result exact and the caller divides by K).
 *
 * The steps follow the paper's order: the corner turn and the widening of
 * 4-bit samples (Sec. 2.4, the unpacking step), then the cross multiplication.  Both
 * are written as plain loops; channels are independent (Sec. 2.1: the X-stage
 * is parallel in frequency) and are spread over POSIX threads.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { XO_CI4 = 0, XO_CI8 = 1, XO_CF32 = 2 };

/* 4-bit two's-complement value of the low four bits of v. */
static int nibble_value(unsigned v)
{
    v &= 15u;
    return (v >= 8u) ? (int)v - 16 : (int)v;
}

/* Sec. 2.3 / Sec. 4: each complex sample is 4 bits real and 4 bits imaginary.
 * Reading: real in the high nibble, imaginary in the low nibble. */
void xo_decode_ci4(uint8_t b, int *re, int *im)
{
    *re = nibble_value((unsigned)b >> 4);
    *im = nibble_value((unsigned)b);
}

/* The unpack and corner turn for one channel: sample (t, c, i) of the input
 * is widened and stored at [i][t] of two planes (real and imaginary). */
static void corner_turn_int(int fmt, const void *in, int64_t n_time, int n_chan,
                            int n_inputs, int c, int64_t *xr, int64_t *xi)
{
    for (int64_t t = 0; t < n_time; ++t) {
        for (int i = 0; i < n_inputs; ++i) {
            int64_t s = (t * n_chan + c) * (int64_t)n_inputs + i;
            int re, im;
            if (fmt == XO_CI4) {
                xo_decode_ci4(((const uint8_t *)in)[s], &re, &im);
            } else {
                re = ((const int8_t *)in)[2 * s];
                im = ((const int8_t *)in)[2 * s + 1];
            }
            xr[(int64_t)i * n_time + t] = re;
            xi[(int64_t)i * n_time + t] = im;
        }
    }
}

static void corner_turn_f64(const float *in, int64_t n_time, int n_chan, int n_inputs,
                            int c, double *xr, double *xi)
{
    for (int64_t t = 0; t < n_time; ++t) {
        for (int i = 0; i < n_inputs; ++i) {
            int64_t s = (t * n_chan + c) * (int64_t)n_inputs + i;
            xr[(int64_t)i * n_time + t] = (double)in[2 * s];
            xi[(int64_t)i * n_time + t] = (double)in[2 * s + 1];
        }
    }
}

/* Cross multiply and integrate one channel: out[pair][2]. */
static void cross_multiply_int(const int64_t *xr, const int64_t *xi, int64_t n_time,
                               int n_inputs, int64_t *out)
{
    for (int i = 0; i < n_inputs; ++i) {
        const int64_t *ri = xr + (int64_t)i * n_time, *mi = xi + (int64_t)i * n_time;
        for (int j = 0; j <= i; ++j) {
            const int64_t *rj = xr + (int64_t)j * n_time, *mj = xi + (int64_t)j * n_time;
            int64_t re = 0, im = 0;
            for (int64_t t = 0; t < n_time; ++t) {
                re += ri[t] * rj[t] + mi[t] * mj[t];
                im += mi[t] * rj[t] - ri[t] * mj[t];
            }
            int64_t p = (int64_t)i * (i + 1) / 2 + j;
            out[2 * p] = re;
            out[2 * p + 1] = im;
        }
    }
}

static void cross_multiply_f64(const double *xr, const double *xi, int64_t n_time,
                               int n_inputs, double *out)
{
    for (int i = 0; i < n_inputs; ++i) {
        const double *ri = xr + (int64_t)i * n_time, *mi = xi + (int64_t)i * n_time;
        for (int j = 0; j <= i; ++j) {
            const double *rj = xr + (int64_t)j * n_time, *mj = xi + (int64_t)j * n_time;
            double re = 0.0, im = 0.0;
            for (int64_t t = 0; t < n_time; ++t) {
                re += ri[t] * rj[t] + mi[t] * mj[t];
                im += mi[t] * rj[t] - ri[t] * mj[t];
            }
            int64_t p = (int64_t)i * (i + 1) / 2 + j;
            out[2 * p] = re;
            out[2 * p + 1] = im;
        }
    }
}

struct job {
    int fmt;
    const void *in;
    int64_t n_time;
    int n_chan, n_inputs, c0, c1, stride, first;
    void *out;
    int failed;
};

static void *run_job(void *arg)
{
    struct job *jb = (struct job *)arg;
    int64_t plane = (int64_t)jb->n_inputs * (jb->n_time > 0 ? jb->n_time : 1);
    int64_t n_pairs = (int64_t)jb->n_inputs * (jb->n_inputs + 1) / 2;
    int is_float = (jb->fmt == XO_CF32);
    void *xr = malloc((size_t)plane * 8), *xi = malloc((size_t)plane * 8);
    if (!xr || !xi) {
        jb->failed = 1;
        free(xr);
        free(xi);
        return NULL;
    }
    for (int c = jb->c0 + jb->first; c < jb->c1; c += jb->stride) {
        int64_t off = (int64_t)(c - jb->c0) * n_pairs * 2;
        if (is_float) {
            corner_turn_f64((const float *)jb->in, jb->n_time, jb->n_chan, jb->n_inputs, c,
                            (double *)xr, (double *)xi);
            cross_multiply_f64((const double *)xr, (const double *)xi, jb->n_time,
                               jb->n_inputs, (double *)jb->out + off);
        } else {
            corner_turn_int(jb->fmt, jb->in, jb->n_time, jb->n_chan, jb->n_inputs, c,
                            (int64_t *)xr, (int64_t *)xi);
            cross_multiply_int((const int64_t *)xr, (const int64_t *)xi, jb->n_time,
                               jb->n_inputs, (int64_t *)jb->out + off);
        }
    }
    free(xr);
    free(xi);
    return NULL;
}

/*
 * Correlate channels [c0, c1) of an input of n_time samples.  `in` is CI4
 * (uint8, one byte per sample), CI8 (int8 re, im) or CF32 (float re, im), in
 * [time][channel][input] order with n_inputs = 2 * stations.  `out` receives
 * (c1 - c0) * P * 2 values: int64 for CI4/CI8, double for CF32.  Returns 0 on
 * success, -1 on bad arguments, -2 when memory runs out.
 */
int xo_correlate(int fmt, const void *in, int64_t n_time, int n_chan, int n_inputs,
                 int c0, int c1, void *out, int n_threads)
{
    if (fmt < XO_CI4 || fmt > XO_CF32 || n_time < 0 || n_inputs < 1 || c0 < 0 ||
        c1 > n_chan || c0 > c1 || (!in && n_time > 0) || !out)
        return -1;
    if (n_threads < 1)
        n_threads = 1;
    if (n_threads > c1 - c0)
        n_threads = (c1 - c0) > 0 ? (c1 - c0) : 1;
    struct job *jobs = (struct job *)calloc((size_t)n_threads, sizeof(struct job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return -2;
    }
    int rc = 0;
    for (int k = 0; k < n_threads; ++k) {
        jobs[k] = (struct job){fmt, in, n_time, n_chan, n_inputs, c0, c1, n_threads, k, out, 0};
        if (n_threads == 1 || pthread_create(&tid[k], NULL, run_job, &jobs[k]) != 0) {
            tid[k] = 0;
            run_job(&jobs[k]);
        }
    }
    for (int k = 0; k < n_threads; ++k) {
        if (tid[k])
            pthread_join(tid[k], NULL);
        if (jobs[k].failed)
            rc = -2;
    }
    free(jobs);
    free(tid);
    return rc;
}

/*
 * Single visibilities, computed one by one straight from the packed input:
 * entry k is channel trip[3k], inputs i = trip[3k+1] >= j = trip[3k+2].
 * out[2k], out[2k+1] receive (re, im), int64 for integer formats and double
 * for CF32.  Returns 0, or -1 on a bad argument (the offending entry is not
 * written).
 */
int xo_correlate_pairs(int fmt, const void *in, int64_t n_time, int n_chan, int n_inputs,
                       const int64_t *trip, int64_t n, void *out)
{
    if (fmt < XO_CI4 || fmt > XO_CF32 || n_time < 0 || n_inputs < 1 || !trip || !out)
        return -1;
    for (int64_t k = 0; k < n; ++k) {
        int64_t c = trip[3 * k], i = trip[3 * k + 1], j = trip[3 * k + 2];
        if (c < 0 || c >= n_chan || i < 0 || i >= n_inputs || j < 0 || j > i)
            return -1;
        int64_t sre = 0, sim = 0;
        double fre = 0.0, fim = 0.0;
        for (int64_t t = 0; t < n_time; ++t) {
            int64_t si = (t * n_chan + c) * (int64_t)n_inputs + i;
            int64_t sj = (t * n_chan + c) * (int64_t)n_inputs + j;
            if (fmt == XO_CF32) {
                const float *f = (const float *)in;
                double ar = f[2 * si], ai = f[2 * si + 1], br = f[2 * sj], bi = f[2 * sj + 1];
                fre += ar * br + ai * bi;
                fim += ai * br - ar * bi;
            } else {
                int ar, ai, br, bi;
                if (fmt == XO_CI4) {
                    xo_decode_ci4(((const uint8_t *)in)[si], &ar, &ai);
                    xo_decode_ci4(((const uint8_t *)in)[sj], &br, &bi);
                } else {
                    const int8_t *b = (const int8_t *)in;
                    ar = b[2 * si];
                    ai = b[2 * si + 1];
                    br = b[2 * sj];
                    bi = b[2 * sj + 1];
                }
                sre += (int64_t)ar * br + (int64_t)ai * bi;
                sim += (int64_t)ai * br - (int64_t)ar * bi;
            }
        }
        if (fmt == XO_CF32) {
            ((double *)out)[2 * k] = fre;
            ((double *)out)[2 * k + 1] = fim;
        } else {
            ((int64_t *)out)[2 * k] = sre;
            ((int64_t *)out)[2 * k + 1] = sim;
        }
    }
    return 0;
}
