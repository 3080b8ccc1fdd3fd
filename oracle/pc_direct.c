/*
 * Direct-summation apply of the product-convolution operator (oracle; test
 * infrastructure only).
 *
 *   (A~ f)[y] = sum_k (phi_k^E * (w_k . f))[y]                 Eq. conv_op_approx_main
 *   (psi * g)[y] = sum_x g[x] psi[y - x]                         Eq. convolution_definition
 *
 * with w_k supported on bbox(U_k) (zero outside U_k) and phi_k^E supported on
 * the window [-R, R]^d, both extended by zero elsewhere.  For each output y
 * (in the order given), for k ascending, for x in bbox(U_k) with y - x in the
 * window (x in row-major order):  acc += (w_k[x] * f[x]) * phi_k^E[y - x].
 * FP64 throughout; OpenMP parallelises over output points only, so every sum
 * is formed in one fixed order whatever the thread count.
 *
 * Everything is handled as 3D: 1D/2D problems pass leading extents of 1 and a
 * window of extent 1 on those axes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

int pc_oracle_apply(const int64_t *shape,   /* [3] */
                    int32_t r,
                    const int64_t *bb_lo,   /* [r][3] */
                    const int64_t *bb_hi,   /* [r][3] */
                    const int64_t *w_off,   /* [r]: offset of w_k on bbox(U_k) in w */
                    const double *w,
                    const int64_t *win,     /* [3]: window extents (odd) */
                    const double *phiE,     /* [r][win0*win1*win2] */
                    int32_t nrhs,
                    const double *f,        /* [nrhs][N] */
                    int64_t ny,
                    const int64_t *ylist,   /* [ny] flat indices, or NULL for all N in order */
                    double *out,            /* [nrhs][ny] */
                    int32_t nthreads)
{
    const int64_t n0 = shape[0], n1 = shape[1], n2 = shape[2];
    const int64_t N = n0 * n1 * n2;
    const int64_t h0 = (win[0] - 1) / 2, h1 = (win[1] - 1) / 2, h2 = (win[2] - 1) / 2;
    const int64_t wsz = win[0] * win[1] * win[2];
    double *ft = (double *)malloc(sizeof(double) * (size_t)N * (size_t)nrhs);
    if (!ft) return 1;
    for (int64_t b = 0; b < nrhs; ++b)
        for (int64_t i = 0; i < N; ++i) ft[i * nrhs + b] = f[b * N + i];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int failed = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)nrhs);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < ny; ++t) {
            if (!acc) continue;
            const int64_t iy = ylist ? ylist[t] : t;
            const int64_t y0 = iy / (n1 * n2), y1 = (iy / n2) % n1, y2 = iy % n2;
            for (int b = 0; b < nrhs; ++b) acc[b] = 0.0;
            for (int32_t k = 0; k < r; ++k) {
                const int64_t *lo = bb_lo + 3 * k, *hi = bb_hi + 3 * k;
                const int64_t a0 = imax64(lo[0], y0 - h0), e0 = imin64(hi[0], y0 + h0);
                const int64_t a1 = imax64(lo[1], y1 - h1), e1 = imin64(hi[1], y1 + h1);
                const int64_t a2 = imax64(lo[2], y2 - h2), e2 = imin64(hi[2], y2 + h2);
                if (a0 > e0 || a1 > e1 || a2 > e2) continue;
                const int64_t m1 = hi[1] - lo[1] + 1, m2 = hi[2] - lo[2] + 1;
                const double *wk = w + w_off[k];
                const double *pk = phiE + (int64_t)k * wsz;
                for (int64_t x0 = a0; x0 <= e0; ++x0)
                    for (int64_t x1 = a1; x1 <= e1; ++x1)
                        for (int64_t x2 = a2; x2 <= e2; ++x2) {
                            const double wv = wk[((x0 - lo[0]) * m1 + (x1 - lo[1])) * m2 + (x2 - lo[2])];
                            const double pv = pk[((y0 - x0 + h0) * win[1] + (y1 - x1 + h1)) * win[2] + (y2 - x2 + h2)];
                            const double *fx = ft + ((x0 * n1 + x1) * n2 + x2) * nrhs;
                            for (int b = 0; b < nrhs; ++b) acc[b] += (wv * fx[b]) * pv;
                        }
            }
            for (int b = 0; b < nrhs; ++b) out[(int64_t)b * ny + t] = acc[b];
        }
        free(acc);
    }
    free(ft);
    return failed;
}

/*
 * Direct-summation apply of the adjoint (oracle; test infrastructure only).
 *
 *   (A~* f)[x] = sum_k w_k[x] (flip(phi_k^E) * f)[x]          Eq. adjoint_random_z
 *              = sum_k w_k[x] sum_y phi_k^E[y - x] f[y]         (real data)
 *
 * For each output x (in the order given), for k ascending with x in
 * bbox(U_k): the correlation sum over y in Omega with y - x in the window
 * (y in row-major order) is formed first, then multiplied by w_k[x] and
 * added.  FP64; OpenMP over output points only.
 */
int pc_oracle_apply_adjoint(const int64_t *shape, int32_t r, const int64_t *bb_lo, const int64_t *bb_hi,
                            const int64_t *w_off, const double *w, const int64_t *win, const double *phiE,
                            int32_t nrhs, const double *f, int64_t nx, const int64_t *xlist, double *out,
                            int32_t nthreads)
{
    const int64_t n0 = shape[0], n1 = shape[1], n2 = shape[2];
    const int64_t N = n0 * n1 * n2;
    const int64_t h0 = (win[0] - 1) / 2, h1 = (win[1] - 1) / 2, h2 = (win[2] - 1) / 2;
    const int64_t wsz = win[0] * win[1] * win[2];
    double *ft = (double *)malloc(sizeof(double) * (size_t)N * (size_t)nrhs);
    if (!ft) return 1;
    for (int64_t b = 0; b < nrhs; ++b)
        for (int64_t i = 0; i < N; ++i) ft[i * nrhs + b] = f[b * N + i];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int failed = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)nrhs);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nx; ++t) {
            if (!acc) continue;
            double *sum = acc + nrhs;
            const int64_t ix = xlist ? xlist[t] : t;
            const int64_t x0 = ix / (n1 * n2), x1 = (ix / n2) % n1, x2 = ix % n2;
            for (int b = 0; b < nrhs; ++b) acc[b] = 0.0;
            for (int32_t k = 0; k < r; ++k) {
                const int64_t *lo = bb_lo + 3 * k, *hi = bb_hi + 3 * k;
                if (x0 < lo[0] || x0 > hi[0] || x1 < lo[1] || x1 > hi[1] || x2 < lo[2] || x2 > hi[2]) continue;
                const int64_t m1 = hi[1] - lo[1] + 1, m2 = hi[2] - lo[2] + 1;
                const double wv = w[w_off[k] + ((x0 - lo[0]) * m1 + (x1 - lo[1])) * m2 + (x2 - lo[2])];
                const double *pk = phiE + (int64_t)k * wsz;
                const int64_t a0 = imax64(0, x0 - h0), e0 = imin64(n0 - 1, x0 + h0);
                const int64_t a1 = imax64(0, x1 - h1), e1 = imin64(n1 - 1, x1 + h1);
                const int64_t a2 = imax64(0, x2 - h2), e2 = imin64(n2 - 1, x2 + h2);
                for (int b = 0; b < nrhs; ++b) sum[b] = 0.0;
                for (int64_t y0 = a0; y0 <= e0; ++y0)
                    for (int64_t y1 = a1; y1 <= e1; ++y1)
                        for (int64_t y2 = a2; y2 <= e2; ++y2) {
                            const double pv = pk[((y0 - x0 + h0) * win[1] + (y1 - x1 + h1)) * win[2] + (y2 - x2 + h2)];
                            const double *fy = ft + ((y0 * n1 + y1) * n2 + y2) * nrhs;
                            for (int b = 0; b < nrhs; ++b) sum[b] += pv * fy[b];
                        }
                for (int b = 0; b < nrhs; ++b) acc[b] += wv * sum[b];
            }
            for (int b = 0; b < nrhs; ++b) out[(int64_t)b * nx + t] = acc[b];
        }
        free(acc);
    }
    free(ft);
    return failed;
}
