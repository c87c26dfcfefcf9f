// Correction Step (Section 2.3, Algorithm convgridding; Section 3.3.8) and the
// centre/corner origin shift used around the FFT (Section 3.3.6).
//
//   correct: image[pol][i][j] *= s(i, j) h(m_i) h(l_j), s = (-1)^(i+j) when the
//            image comes from (or goes to) an FFT of a shifted grid, else 1.
//   shift:   grid[pol][kv][ku] *= (-1)^(kv+ku).
//   fold:    grid += err, err = 0 (ends a compensated gridding sequence).
// For even N, (-1)^(k) before and (-1)^(i) after an unnormalised FFT turn it
// into the transform with both origins at pixel N/2.
#include "gw_internal.cuh"

namespace gw {

namespace {

__global__ void k_correct(float2* __restrict__ img, const float* __restrict__ h, int N, int npol,
                          int shift) {
    const int64_t n = (int64_t)N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e - (int64_t)i * N);
        float m = __ldg(h + i) * __ldg(h + j);
        if (shift && ((i + j) & 1)) m = -m;
        for (int p = 0; p < npol; ++p) {
            float2 v = img[(int64_t)p * n + e];
            v.x *= m;
            v.y *= m;
            img[(int64_t)p * n + e] = v;
        }
    }
}

__global__ void k_shift(float2* __restrict__ g, int N, int npol) {
    const int64_t n = (int64_t)N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e - (int64_t)i * N);
        if (!((i + j) & 1)) continue;
        for (int p = 0; p < npol; ++p) {
            float2 v = g[(int64_t)p * n + e];
            g[(int64_t)p * n + e] = make_float2(-v.x, -v.y);
        }
    }
}

__global__ void k_fold(float2* __restrict__ g, float2* __restrict__ err, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float2 d = err[e];
        if (d.x == 0.f && d.y == 0.f) continue;
        float2 v = g[e];
        v.x += d.x;
        v.y += d.y;
        g[e] = v;
        err[e] = make_float2(0.f, 0.f);
    }
}

__global__ void k_zero_vis(uint32_t* __restrict__ v, int64_t n_max, int words, DevCount dc) {
    const int64_t n = dc.clamp(n_max) * words;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        v[e] = 0u;
}

// Sum of layer images times their w-screens (w-stacking, Section 1.7.1):
// the screen of layer l at pixel (i, j) is exp(+j 2 pi w_l (n - 1)) with
// n - 1 = -r^2 / (1 + sqrt(1 - r^2)), r^2 = l_j^2 + m_i^2; it is formed in
// FP64 as screen_0 * rot^l, rot = exp(+j 2 pi dw (n - 1)).
// exp(+j pi a) for a phase a in units of pi: a is reduced to [-1, 1] in FP64
// (exact for the |a| of any w-screen), then evaluated in FP32.
__device__ __forceinline__ void screen_pi(double a, float& s, float& c) {
    const double r = a - 2.0 * rint(0.5 * a);
    sincospif((float)r, &s, &c);
}

// Sum of the layer images times their w-screens exp(+j 2 pi w_l (n - 1)),
// w_l = wmin + l dw.  n - 1 is computed in FP64 (w (n - 1) reaches hundreds
// of radians); the screens follow a rotation recursion in FP32 from an
// anchor recomputed every 8 layers, and the sum is FP32.  The layer images
// are the inverse transforms of the unshifted layer grids: the centring
// factor (-1)^(u + v) of the grid is the circular shift by N/2 of its
// transform, applied here in the read (N is even).  One thread per pixel;
// the layers are read once, coalesced, so the kernel is HBM bound.
__global__ void k_wstack_combine(const float2* __restrict__ layers, int nlayers, double wmin,
                                 double dw, int N, int npol, double cell,
                                 float2* __restrict__ image) {
    const int64_t n = (int64_t)N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e - (int64_t)i * N);
        const double l = (j - N / 2) * cell, m = (i - N / 2) * cell;
        const double r2 = l * l + m * m;
        const double nm1 = r2 < 1.0 ? -r2 / (1.0 + sqrt(1.0 - r2)) : 0.0;
        const int is = i + N / 2 < N ? i + N / 2 : i - N / 2;
        const int js = j + N / 2 < N ? j + N / 2 : j - N / 2;
        const int64_t es = (int64_t)is * N + js;      // pixel of the unshifted transform
        float s1, c1;                                 // one layer step
        screen_pi(2.0 * dw * nm1, s1, c1);
        float acc[4][2] = {};
        float cr = 1.f, ci = 0.f;
        for (int L = 0; L < nlayers; ++L) {
            if ((L & 7) == 0) screen_pi(2.0 * (wmin + L * dw) * nm1, ci, cr);
            for (int p = 0; p < npol && p < 4; ++p) {
                const float2 v = __ldcs(layers + ((int64_t)L * npol + p) * n + es);
                acc[p][0] = fmaf(v.x, cr, fmaf(-v.y, ci, acc[p][0]));
                acc[p][1] = fmaf(v.x, ci, fmaf(v.y, cr, acc[p][1]));
            }
            const float nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
            cr = nr;
            ci = ni;
        }
        for (int p = 0; p < npol && p < 4; ++p) {
            float2 o = image[(int64_t)p * n + e];
            o.x += acc[p][0];
            o.y += acc[p][1];
            image[(int64_t)p * n + e] = o;
        }
    }
}

unsigned blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > current_sm_count() * 32) b = current_sm_count() * 32;
    return (unsigned)std::max<int64_t>(b, 1);
}

}  // namespace

void launch_correct(float2* image, const float* h, int N, int npol, int mode, cudaStream_t s) {
    k_correct<<<blocks_for((int64_t)N * N), 256, 0, s>>>(image, h, N, npol, mode != 0);
    note_launch();
}

void launch_shift(float2* grid, int N, int npol, cudaStream_t s) {
    k_shift<<<blocks_for((int64_t)N * N), 256, 0, s>>>(grid, N, npol);
    note_launch();
}

void launch_zero_vis(void* vis, int kind, int64_t n_max, int npol, DevCount dc, cudaStream_t s) {
    const int words = npol * dtype_bytes(kind) / 4;
    k_zero_vis<<<blocks_for(n_max * words), 256, 0, s>>>(static_cast<uint32_t*>(vis), n_max, words,
                                                        dc);
    note_launch();
}

void launch_wstack_combine(const float2* layers, int nlayers, double wmin, double dw, int N,
                           int npol, double cell, float2* image, cudaStream_t s) {
    k_wstack_combine<<<blocks_for((int64_t)N * N), 256, 0, s>>>(layers, nlayers, wmin, dw, N, npol,
                                                                 cell, image);
    note_launch();
}

void launch_fold(float2* grid, float2* err, int64_t n, cudaStream_t s) {
    k_fold<<<blocks_for(n), 256, 0, s>>>(grid, err, n);
    note_launch();
}

}  // namespace gw
