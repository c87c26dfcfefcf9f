/*
 * Plain FP64 gridding and degridding loops.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the CPU-baseline leg of
 * the benchmark, never by the product library.  Compiled with
 * -ffp-contract=off so every multiply and add is a separate IEEE operation.
 *
 * Gridding (Section 2.4.5, Algorithm convgriddingoversampling, Gridding
 * Step, with the w-projection GCF of Section 1.7.1): for every valid record
 * i with pixel (kv, ku), oversampled offset (ov, ou), plane p and value V,
 *
 *     G[pol][kv + tv][ku + tu] += K_i(tv, tu) * (V[pol] * weight[pol])
 *
 * for all taps |tv|, |tu| <= h_p, where K_i is the table slice
 * K_p[ov][ou] or its complex conjugate when the record has w < 0.
 *
 * Degridding (the adjoint of the above, unweighted):
 *
 *     V[pol] = sum_{tv, tu} conj(K_i(tv, tu)) * G[pol][kv + tv][ku + tu].
 *
 * Complex numbers are interleaved (re, im) doubles.  The table of plane p
 * starts at table + 2 * plane_off[p] and is laid out
 * [ov + beta/2][ou + beta/2][tv + h][tu + h].
 *
 * Parallelism: gridding splits the grid rows into bands, one per thread;
 * every thread scans all records in order and applies only the taps that
 * land in its band, so each grid point receives its contributions in record
 * order, exactly as in the serial loop.  Degridding parallelises over
 * records, which are independent.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void grid_band(int r0, int r1, int N, int npol, int beta,
                      const int32_t* support, const int64_t* plane_off, const double* table,
                      int64_t nvis, const int32_t* ku, const int32_t* kv, const int32_t* ou,
                      const int32_t* ov, const int32_t* plane, const uint8_t* flags,
                      const double* vis, const double* weight, double* grid)
{
    for (int64_t i = 0; i < nvis; ++i) {
        if (!(flags[i] & 1)) continue;
        const int p = plane[i];
        const int S = support[p];
        const int h = (S - 1) / 2;
        const int vlo = kv[i] - h, vhi = kv[i] + h;
        if (vhi < r0 || vlo >= r1) continue;
        const int conj = (flags[i] & 2) != 0;
        const double* K = table + 2 * (plane_off[p] +
            ((int64_t)(ov[i] + beta / 2) * beta + (ou[i] + beta / 2)) * (int64_t)S * S);
        for (int pol = 0; pol < npol; ++pol) {
            double vr = vis[2 * (i * npol + pol)];
            double vi = vis[2 * (i * npol + pol) + 1];
            if (weight) {
                const double wt = weight[i * npol + pol];
                vr = vr * wt;
                vi = vi * wt;
            }
            double* G = grid + 2 * (int64_t)pol * N * N;
            for (int tv = -h; tv <= h; ++tv) {
                const int row = kv[i] + tv;
                if (row < r0 || row >= r1) continue;
                for (int tu = -h; tu <= h; ++tu) {
                    const double* k = K + 2 * ((int64_t)(tv + h) * S + (tu + h));
                    const double kr = k[0];
                    const double ki = conj ? -k[1] : k[1];
                    double* g = G + 2 * ((int64_t)row * N + (ku[i] + tu));
                    g[0] = g[0] + (kr * vr - ki * vi);
                    g[1] = g[1] + (kr * vi + ki * vr);
                }
            }
        }
    }
}

int oracle_grid(int N, int npol, int beta, const int32_t* support, const int64_t* plane_off,
                const double* table, int64_t nvis, const int32_t* ku, const int32_t* kv,
                const int32_t* ou, const int32_t* ov, const int32_t* plane,
                const uint8_t* flags, const double* vis, const double* weight, double* grid,
                int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N) nthreads = N;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
#endif
    for (int b = 0; b < nthreads; ++b) {
        const int r0 = (int)((int64_t)N * b / nthreads);
        const int r1 = (int)((int64_t)N * (b + 1) / nthreads);
        grid_band(r0, r1, N, npol, beta, support, plane_off, table, nvis, ku, kv, ou, ov,
                  plane, flags, vis, weight, grid);
    }
    return 0;
}

int oracle_degrid(int N, int npol, int beta, const int32_t* support, const int64_t* plane_off,
                  const double* table, int64_t nvis, const int32_t* ku, const int32_t* kv,
                  const int32_t* ou, const int32_t* ov, const int32_t* plane,
                  const uint8_t* flags, const double* grid, double* vis_out, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 256)
#endif
    for (int64_t i = 0; i < nvis; ++i) {
        for (int pol = 0; pol < npol; ++pol) {
            vis_out[2 * (i * npol + pol)] = 0.0;
            vis_out[2 * (i * npol + pol) + 1] = 0.0;
        }
        if (!(flags[i] & 1)) continue;
        const int p = plane[i];
        const int S = support[p];
        const int h = (S - 1) / 2;
        const int conj = (flags[i] & 2) != 0;
        const double* K = table + 2 * (plane_off[p] +
            ((int64_t)(ov[i] + beta / 2) * beta + (ou[i] + beta / 2)) * (int64_t)S * S);
        for (int pol = 0; pol < npol; ++pol) {
            const double* G = grid + 2 * (int64_t)pol * N * N;
            double sr = 0.0, si = 0.0;
            for (int tv = -h; tv <= h; ++tv) {
                for (int tu = -h; tu <= h; ++tu) {
                    const double* k = K + 2 * ((int64_t)(tv + h) * S + (tu + h));
                    /* the record's kernel is K (or conj K for w < 0); the adjoint
                       multiplies by its conjugate */
                    const double kr = k[0];
                    const double ki = conj ? k[1] : -k[1];
                    const double* g = G + 2 * ((int64_t)(kv[i] + tv) * N + (ku[i] + tu));
                    sr = sr + (kr * g[0] - ki * g[1]);
                    si = si + (kr * g[1] + ki * g[0]);
                }
            }
            vis_out[2 * (i * npol + pol)] = sr;
            vis_out[2 * (i * npol + pol) + 1] = si;
        }
    }
    return 0;
}

/*
 * Gridding evaluated only at the lattice points (off + step * a, off + step * b),
 * a, b = 0 .. m-1, for full-size checks: out[pol][b][a] (row = v) receives the
 * same sum as the full grid at that point, accumulated in record order.
 */
int oracle_grid_lattice(int N, int npol, int beta, const int32_t* support,
                        const int64_t* plane_off, const double* table, int64_t nvis,
                        const int32_t* ku, const int32_t* kv, const int32_t* ou,
                        const int32_t* ov, const int32_t* plane, const uint8_t* flags,
                        const double* vis, const double* weight, int off, int step, int m,
                        double* out)
{
    (void)N;
    for (int64_t i = 0; i < nvis; ++i) {
        if (!(flags[i] & 1)) continue;
        const int p = plane[i];
        const int S = support[p];
        const int h = (S - 1) / 2;
        const int conj = (flags[i] & 2) != 0;
        /* lattice indices whose point lies in [k - h, k + h] */
        int a0 = (ku[i] - h - off + step - 1) / step, a1 = (ku[i] + h - off) / step;
        int b0 = (kv[i] - h - off + step - 1) / step, b1 = (kv[i] + h - off) / step;
        if (ku[i] - h - off < 0) a0 = 0;
        if (kv[i] - h - off < 0) b0 = 0;
        if (ku[i] + h - off < 0 || kv[i] + h - off < 0) continue;
        if (a1 > m - 1) a1 = m - 1;
        if (b1 > m - 1) b1 = m - 1;
        const double* K = table + 2 * (plane_off[p] +
            ((int64_t)(ov[i] + beta / 2) * beta + (ou[i] + beta / 2)) * (int64_t)S * S);
        for (int b = b0; b <= b1; ++b) {
            const int tv = off + step * b - kv[i];
            for (int a = a0; a <= a1; ++a) {
                const int tu = off + step * a - ku[i];
                const double* k = K + 2 * ((int64_t)(tv + h) * S + (tu + h));
                const double kr = k[0];
                const double ki = conj ? -k[1] : k[1];
                for (int pol = 0; pol < npol; ++pol) {
                    double vr = vis[2 * (i * npol + pol)];
                    double vi = vis[2 * (i * npol + pol) + 1];
                    if (weight) {
                        const double wt = weight[i * npol + pol];
                        vr = vr * wt;
                        vi = vi * wt;
                    }
                    double* g = out + 2 * (((int64_t)pol * m + b) * m + a);
                    g[0] = g[0] + (kr * vr - ki * vi);
                    g[1] = g[1] + (kr * vi + ki * vr);
                }
            }
        }
    }
    return 0;
}
