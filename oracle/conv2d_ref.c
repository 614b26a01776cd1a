/*
 * Oracle: plain FP64 direct 2-D cross-correlation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's shared object.  It shares no code,
 * header or constant with the CUDA path.
 *
 * The operation (the paper never defines the convolution; the workload is an
 * FP32 2-D convolution with a zero-padded input, read as a cross-correlation
 * with no filter flip):
 *
 *     ref[y][x] = sum_{j=0}^{fh-1} sum_{i=0}^{fw-1} in[y+j][x+i] * filt[j][i]
 *
 * for 0 <= y < out_h = in_h - fh + 1 and 0 <= x < out_w = in_w - fw + 1, with
 * every product and sum taken in double precision.  `in` is the padded input
 * (row pitch `in_pitch` elements), so "same"-size output comes from an input
 * padded by (fh-1)/2 and (fw-1)/2 zeros per side, done by the caller.
 *
 * Plain loops, no blocking and no reordering: j outer, i inner, one running
 * double sum per output.  OpenMP splits the output rows across threads.
 */
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_conv2d_f64(const float *in, long in_pitch, long in_h, long in_w,
                      const float *filt, long fh, long fw,
                      double *out, long out_pitch, long out_h, long out_w,
                      int nthreads)
{
    if (!in || !filt || !out) return -1;
    if (fh < 1 || fw < 1 || in_h < fh || in_w < fw) return -1;
    if (out_h != in_h - fh + 1 || out_w != in_w - fw + 1) return -1;
    if (in_pitch < in_w || out_pitch < out_w) return -1;
    if (nthreads < 1) nthreads = 1;

    long y;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (y = 0; y < out_h; ++y) {
        for (long x = 0; x < out_w; ++x) {
            double s = 0.0;
            for (long j = 0; j < fh; ++j) {
                const float *row = in + (y + j) * in_pitch + x;
                const float *frow = filt + j * fw;
                for (long i = 0; i < fw; ++i)
                    s += (double)row[i] * (double)frow[i];
            }
            out[y * out_pitch + x] = s;
        }
    }
    return 0;
}

/*
 * The same sum evaluated only at n chosen output coordinates (ys[k], xs[k]);
 * used to check sampled outputs of full-size problems one by one.
 */
int oracle_conv2d_points_f64(const float *in, long in_pitch, long in_h, long in_w,
                             const float *filt, long fh, long fw,
                             const long *ys, const long *xs, long n,
                             double *out, int nthreads)
{
    if (!in || !filt || !ys || !xs || !out) return -1;
    if (fh < 1 || fw < 1 || in_h < fh || in_w < fw || in_pitch < in_w) return -1;
    for (long k = 0; k < n; ++k)
        if (ys[k] < 0 || xs[k] < 0 || ys[k] > in_h - fh || xs[k] > in_w - fw) return -1;
    if (nthreads < 1) nthreads = 1;

    long k;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (k = 0; k < n; ++k) {
        double s = 0.0;
        for (long j = 0; j < fh; ++j)
            for (long i = 0; i < fw; ++i)
                s += (double)in[(ys[k] + j) * in_pitch + xs[k] + i] * (double)filt[j * fw + i];
        out[k] = s;
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
