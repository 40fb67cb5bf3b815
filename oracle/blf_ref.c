/*
 * TEST INFRASTRUCTURE ONLY -- the FP64 reference ("oracle") bilateral filter.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg load this file's
 * shared library.  The CUDA product path shares no code with it.
 *
 * Definition followed (Section II-A, Eq. 1): for every pixel s of a field g,
 *     v_s = (1/Z_s) * sum_{t in N(s)} G_ss(|s-t|) * G_sr(|g_s-g_t|) * g_t,
 *     Z_s = sum_{t in N(s)} G_ss(|s-t|) * G_sr(|g_s-g_t|),
 * with the readings used throughout this project:
 *   - G_sigma(x) = exp(-x^2 / (2 sigma^2))  (the paper only says "typically Gaussians");
 *   - N(s) is the square window of radius r, (2r+1)^2 taps, centre included;
 *   - indices wrap periodically (the Fourier solve of Eq. 8 already assumes a torus);
 *   - |g_s - g_t| is the scalar difference of one field of one channel;
 *   - sigma_r = +inf means range weight 1 (a truncated spatial Gaussian); sigma_s = +inf means
 *     spatial weight 1.
 * Everything is plain FP64 with libm exp, one pixel at a time, no blocking and no reordering;
 * rows are shared among OpenMP threads.
 */
#include <math.h>
#include <stdlib.h>

static int wrap_index(long i, int n)
{
    long m = i % n;
    return (int)(m < 0 ? m + n : m);
}

/* Bilateral filter of one pixel (y, x).  ws holds the (2r+1)^2 spatial weights. */
static double blf_pixel(const double *g, int H, int W, int r, const double *ws,
                        int range_on, double two_sr2, int y, int x)
{
    const double gs = g[(long)y * W + x];
    double num = 0.0, den = 0.0;
    const int n = 2 * r + 1;
    for (int dy = -r; dy <= r; ++dy) {
        const int yy = wrap_index((long)y + dy, H);
        for (int dx = -r; dx <= r; ++dx) {
            const int xx = wrap_index((long)x + dx, W);
            const double gt = g[(long)yy * W + xx];
            const double diff = gs - gt;
            const double wr = range_on ? exp(-(diff * diff) / two_sr2) : 1.0;
            const double w = ws[(dy + r) * n + (dx + r)] * wr;
            num += w * gt;
            den += w;
        }
    }
    return num / den;
}

static double *spatial_weights(int r, double sigma_s)
{
    const int n = 2 * r + 1;
    double *ws = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!ws) return NULL;
    const int spatial_on = isfinite(sigma_s);
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            const double d2 = (double)(dx * dx + dy * dy);
            ws[(dy + r) * n + (dx + r)] =
                spatial_on ? exp(-d2 / (2.0 * sigma_s * sigma_s)) : 1.0;
        }
    return ws;
}

/* Full field: v = BLF(g).  Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_blf_f64(const double *g, double *v, int H, int W, int r, double sigma_s,
                   double sigma_r, int nthreads)
{
    if (!g || !v || H < 1 || W < 1 || r < 0 || !(sigma_s > 0.0) || !(sigma_r > 0.0))
        return -1;
    double *ws = spatial_weights(r, sigma_s);
    if (!ws) return -1;
    const int range_on = isfinite(sigma_r);
    const double two_sr2 = 2.0 * sigma_r * sigma_r;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            v[(long)y * W + x] = blf_pixel(g, H, W, r, ws, range_on, two_sr2, y, x);
    free(ws);
    return 0;
}

/* Sampled pixels: out[i] = BLF(g) at (ys[i], xs[i]). */
int oracle_blf_at_f64(const double *g, int H, int W, int r, double sigma_s, double sigma_r,
                      const int *ys, const int *xs, int n, double *out, int nthreads)
{
    if (!g || !ys || !xs || !out || H < 1 || W < 1 || r < 0 || n < 0 ||
        !(sigma_s > 0.0) || !(sigma_r > 0.0))
        return -1;
    double *ws = spatial_weights(r, sigma_s);
    if (!ws) return -1;
    const int range_on = isfinite(sigma_r);
    const double two_sr2 = 2.0 * sigma_r * sigma_r;
    int bad = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads) reduction(| : bad)
    for (int i = 0; i < n; ++i) {
        if (ys[i] < 0 || ys[i] >= H || xs[i] < 0 || xs[i] >= W) {
            bad = 1;
            continue;
        }
        out[i] = blf_pixel(g, H, W, r, ws, range_on, two_sr2, ys[i], xs[i]);
    }
    free(ws);
    return bad ? -1 : 0;
}
