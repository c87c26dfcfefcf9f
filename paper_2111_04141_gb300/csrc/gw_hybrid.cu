// Hybrid Gridding with a column pruner (Section 2.4, Algorithm (hybrid)),
// for 2-D plans (no w-term; with w-stacking per layer).
//
//   Gridding Step  k_hybrid_grid: each record is convolved along u with the
//                  oversampled 1-D GCF (S taps) and put on the nearest of
//                  beta N rows along v: fine[pol][q_v][k_u + t] += c(t - o_u/beta) V,
//                  q_v = k_v beta + o_v.  S updates per record instead of S^2.
//   Pruning Step   k_prune: every column is sampled down by beta/2 onto a
//                  2x-oversampled v axis through the pruning GCF Z (S_z taps):
//                  pruned[pol][k][u] = sum_r Z(k - 2r/beta) fine[pol][r][u].
//   IFFT Step      (cuFFT, on the 2N x N pruned grid after k_hybrid_shift).
//   Correction     k_hybrid_image: keep the central N of the 2N rows, re-centre
//                  and apply h_co(l) h_pr(m).
#include "gw_internal.cuh"

namespace gw {

namespace {

unsigned blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)std::max<int64_t>(b, 1);
}

// One thread per (record, tap); consecutive taps of a record are
// consecutive columns of its fine row (coalesced vector atomics).
__global__ void k_hybrid_grid(const gw_index_rec* __restrict__ rec, int64_t nvis,
                              const void* __restrict__ vis, int vis_kind,
                              const float* __restrict__ weight, int npol, int beta, int S,
                              const double* __restrict__ c1, int fmin, double norm, int N, int sz,
                              float2* __restrict__ fine, unsigned long long* __restrict__ dropped) {
    const int h = S / 2, hz = sz / 2;
    const int64_t total = nvis * S;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / S;
        const int t = (int)(e - i * S) - h;
        int4 rv = __ldg(reinterpret_cast<const int4*>(rec) + i);
        const gw_index_rec r = *reinterpret_cast<gw_index_rec*>(&rv);
        if (!(r.flags & GW_FLAG_VALID)) continue;      // counted by the index stage
        const int64_t q = (int64_t)r.kv * beta + r.ov;
        const long long k0 = floor_div(2 * q + beta / 2, beta);
        if (q < 0 || q >= (int64_t)beta * N || k0 - hz < 0 || k0 + hz > 2LL * N - 1) {
            if (t == -h) atomicAdd(dropped, 1ULL);      // pruning window leaves the 2N rows
            continue;
        }
        const float w = (float)(__ldg(c1 + beta * t - r.ou - fmin) / norm);
        const int64_t col = (int64_t)r.ku + t;
        for (int p = 0; p < npol; ++p) {
            float2 v = load_vis(vis, vis_kind, i * npol + p);
            if (weight) {
                const float ww = __ldg(weight + i * npol + p);
                v.x *= ww;
                v.y *= ww;
            }
            atomicAdd(fine + ((int64_t)p * beta * N + q) * N + col, make_float2(w * v.x, w * v.y));
        }
    }
}

// One thread per (pol, output row k, column u): the fine rows whose nearest
// 2x-grid row k0 lies within hz of k, weighted by Z at their offset.
__global__ void k_prune(const float2* __restrict__ fine, int npol, int N, int beta, int sz,
                        const float* __restrict__ z, float2* __restrict__ pruned) {
    const int hz = sz / 2;
    const int64_t rows2 = 2LL * N, fr = (int64_t)beta * N;
    const int64_t total = (int64_t)npol * rows2 * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(e % N);
        const int64_t pk = e / N;
        const int k = (int)(pk % rows2);
        const int p = (int)(pk / rows2);
        // 2r in [(k - hz) beta - beta/2, (k + hz) beta + beta/2)
        const long long lo2 = (long long)(k - hz) * beta - beta / 2;
        const long long hi2 = (long long)(k + hz) * beta + beta / 2;
        long long r0 = (lo2 + 1) >> 1;                       // ceil(lo2 / 2)
        long long r1 = (hi2 + 1) >> 1;                       // ceil(hi2 / 2), exclusive
        if (r0 < 0) r0 = 0;
        if (r1 > fr) r1 = fr;
        float ax = 0.f, ay = 0.f;
        const float2* col = fine + (int64_t)p * fr * N + u;
        for (long long r = r0; r < r1; ++r) {
            const long long k0 = floor_div(2 * r + beta / 2, beta);
            const int o = (int)(2 * r - k0 * beta);
            const float wz = __ldg(z + ((o + beta / 2) / 2) * sz + (k - (int)k0) + hz);
            const float2 f = col[r * N];
            ax = fmaf(wz, f.x, ax);
            ay = fmaf(wz, f.y, ay);
        }
        pruned[e] = make_float2(ax, ay);
    }
}

__global__ void k_hybrid_shift(float2* __restrict__ g, int npol, int N) {
    const int64_t rows2 = 2LL * N;
    const int64_t total = (int64_t)npol * rows2 * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(e % N);
        const int k = (int)((e / N) % rows2);
        if ((k + u) & 1) {
            const float2 v = g[e];
            g[e] = make_float2(-v.x, -v.y);
        }
    }
}

// image[p][i][j] = raw[p][i + N/2][j] (-1)^(i + N/2 + j) (-1)^(N/2) h_pr[i] h_co[j]
__global__ void k_hybrid_image(const float2* __restrict__ raw, int npol, int N,
                               const float* __restrict__ hco, const float* __restrict__ hpr,
                               float2* __restrict__ image) {
    const int64_t total = (int64_t)npol * N * N;
    const int half = N / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % N);
        const int i = (int)((e / N) % N);
        const int p = (int)(e / ((int64_t)N * N));
        float m = __ldg(hco + j) * __ldg(hpr + i);
        if ((i + half + j + half) & 1) m = -m;
        const float2 v = raw[((int64_t)p * 2 * N + i + half) * N + j];
        image[e] = make_float2(v.x * m, v.y * m);
    }
}

}  // namespace

void launch_hybrid_grid(const gw_index_rec* rec, int64_t nvis, const void* vis, int vis_kind,
                        const float* weight, int npol, int beta, int S, const double* c1,
                        int fmin, double norm, int N, int sz, float2* fine,
                        unsigned long long* dropped, cudaStream_t s) {
    if (nvis <= 0) return;
    k_hybrid_grid<<<blocks_for(nvis * S), 256, 0, s>>>(rec, nvis, vis, vis_kind, weight, npol,
                                                       beta, S, c1, fmin, norm, N, sz, fine,
                                                       dropped);
    note_launch();
}

void launch_prune(const float2* fine, int npol, int N, int beta, int sz, const float* z,
                  float2* pruned, cudaStream_t s) {
    k_prune<<<blocks_for((int64_t)npol * 2 * N * N), 256, 0, s>>>(fine, npol, N, beta, sz, z,
                                                                 pruned);
    note_launch();
}

void launch_hybrid_shift(float2* g, int npol, int N, cudaStream_t s) {
    k_hybrid_shift<<<blocks_for((int64_t)npol * 2 * N * N), 256, 0, s>>>(g, npol, N);
    note_launch();
}

void launch_hybrid_image(const float2* raw, int npol, int N, const float* hco, const float* hpr,
                         float2* image, cudaStream_t s) {
    k_hybrid_image<<<blocks_for((int64_t)npol * N * N), 256, 0, s>>>(raw, npol, N, hco, hpr,
                                                                    image);
    note_launch();
}

}  // namespace gw
