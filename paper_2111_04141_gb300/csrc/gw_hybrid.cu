// Hybrid Gridding with a column pruner (Section 2.4, Algorithm (hybrid)),
// for 2-D plans (no w-term; with w-stacking per layer).
//
//   Gridding Step  k_hybrid_grid: each record is convolved along u with the
//                  oversampled 1-D GCF (S taps) and put on the nearest of
//                  beta N rows along v: fine[q_v][k_u + t][pol] += c(t - o_u/beta) V,
//                  q_v = k_v beta + o_v.  S updates per record instead of S^2.
//                  Polarisations are interleaved in the fine grid, so the
//                  updates of one tap are one contiguous 8 npol-byte run
//                  (16-byte vector atomics over polarisation pairs).
//   Pruning Step   k_prune: every column is sampled down by beta/2 onto a
//                  2x-oversampled v axis through the pruning GCF Z (S_z taps):
//                  pruned[pol][k][u] = sum_r Z(k - 2r/beta) fine[r][u][pol];
//                  the pruners see the fine grid as N npol columns
//                  c = u npol + pol and write the planar pruned grid.
//   IFFT Step      (cuFFT, on the 2N x N pruned grid after k_hybrid_shift).
//   Correction     k_hybrid_image: keep the central N of the 2N rows, re-centre
//                  and apply h_co(l) h_pr(m).
#include "gw_internal.cuh"

namespace gw {

namespace {

unsigned blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > current_sm_count() * 32) b = current_sm_count() * 32;
    return (unsigned)std::max<int64_t>(b, 1);
}

// Lanes over (record, tap): a warp takes 32 / S records of S taps at a
// time (S > 32: one record, lanes loop over its taps), so consecutive taps
// of a record are consecutive columns of its fine row (coalesced vector
// atomics).  The 1-D GCF weights c(t - o_u/beta) / norm are rounded to FP32
// once per CTA into a [beta][S] shared table (wtab != 0), not per tap.
__global__ void __launch_bounds__(256) k_hybrid_grid(const gw_index_rec* __restrict__ rec,
                                                     int64_t nvis, const void* __restrict__ vis,
                                                     int vis_kind, const float* __restrict__ weight,
                                                     int npol, int beta, int S,
                                                     const double* __restrict__ c1, int fmin,
                                                     double norm, int N, int sz, int wtab,
                                                     float2* __restrict__ fine,
                                                     unsigned long long* __restrict__ dropped) {
    extern __shared__ float ws[];                          // [beta][S] when wtab
    const int h = S / 2, hz = sz / 2, hb = beta / 2;
    if (wtab) {
        for (int e = threadIdx.x; e < beta * S; e += blockDim.x) {
            const int a = e / S, tt = e - a * S;          // a = o_u + beta/2, tt = t + h
            ws[e] = (float)(c1[beta * (tt - h) - (a - hb) - fmin] / norm);
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int G = S <= 32 ? 32 / S : 1;                    // records per warp pass
    const int rl = S <= 32 ? lane / S : 0;
    const int t0 = S <= 32 ? lane - rl * S : lane;         // first tap (0-based) of this lane
    if (rl >= G) return;                                   // idle lanes (no barriers below)
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp * G + rl; i < nvis; i += nwarps * G) {
        int4 rv = __ldg(reinterpret_cast<const int4*>(rec) + i);
        const gw_index_rec r = *reinterpret_cast<gw_index_rec*>(&rv);
        if (!(r.flags & GW_FLAG_VALID)) continue;          // counted by the index stage
        const int64_t q = (int64_t)r.kv * beta + r.ov;
        const long long k0 = floor_div(2 * q + hb, beta);
        if (q < 0 || q >= (int64_t)beta * N || k0 - hz < 0 || k0 + hz > 2LL * N - 1) {
            if (t0 == 0) atomicAdd(dropped, 1ULL);         // pruning window leaves the 2N rows
            continue;
        }
        for (int tt = t0; tt < S; tt += 32) {
            const int t = tt - h;
            const float w = wtab ? ws[(r.ou + hb) * S + tt]
                                 : (float)(__ldg(c1 + beta * t - r.ou - fmin) / norm);
            float2* dst = fine + ((q * N + r.ku + t) * npol);
            auto wv = [&](int p) {                          // L1 broadcast over the taps
                float2 vv = load_vis(vis, vis_kind, i * npol + p);
                if (weight) {
                    const float ww = __ldg(weight + i * npol + p);
                    vv.x *= ww;
                    vv.y *= ww;
                }
                return make_float2(w * vv.x, w * vv.y);
            };
            int p = 0;
            if (!(npol & 1))                                // 16-byte aligned pairs
                for (; p + 1 < npol; p += 2) {
                    const float2 a = wv(p), b = wv(p + 1);
                    atomicAdd(reinterpret_cast<float4*>(dst + p), make_float4(a.x, a.y, b.x, b.y));
                }
            for (; p < npol; ++p) atomicAdd(dst + p, wv(p));
        }
    }
}

// The fine rows with nearest 2x row k' are r = k' beta/2 - beta/4 + m,
// m = 0 .. beta/2 - 1 (beta % 4 == 0), at offset row m of the Z table; an
// output row k gathers them for k' = k - t, |t| <= hz, with weight Z[m][t + hz].

// One thread per (pol, output row k, column u), reading the fine grid.
__global__ void k_prune(const float2* __restrict__ fine, int npol, int N, int beta, int sz,
                        const float* __restrict__ z, float2* __restrict__ pruned) {
    const int hz = sz / 2, hb = beta / 2;
    const int64_t rows2 = 2LL * N, fr = (int64_t)beta * N;
    const int64_t total = (int64_t)npol * rows2 * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(e % N);
        const int64_t pk = e / N;
        const int k = (int)(pk % rows2);
        const int p = (int)(pk / rows2);
        const int64_t C = (int64_t)N * npol;                    // fine-grid row length
        const float2* col = fine + (int64_t)u * npol + p;
        float ax = 0.f, ay = 0.f;
        for (int t = -hz; t <= hz; ++t) {
            const int64_t rs = (int64_t)(k - t) * hb - beta / 4;
            const int m0 = rs < 0 ? (int)(-rs) : 0;
            const int m1 = rs + hb > fr ? (int)(fr - rs) : hb;
            for (int m = m0; m < m1; ++m) {
                const float wz = __ldg(z + m * sz + t + hz);
                const float2 f = col[(rs + m) * C];
                ax = fmaf(wz, f.x, ax);
                ay = fmaf(wz, f.y, ay);
            }
        }
        pruned[e] = make_float2(ax, ay);
    }
}

// Tiled pruner: a CTA produces R output rows x 32 fine-grid columns
// (c = u npol + pol); the fine rows they need ((R + 2 hz + 1) beta / 2 of them) and
// the Z table are staged in shared memory once, so the fine grid is read
// from memory about once instead of once per output row.
constexpr int kPruneCols = 32;
constexpr int kPruneRowsMax = 352;          // staged fine rows (88 KB of float2 x 32 columns)
constexpr int kPruneZMax = 2048;            // staged Z entries (beta/2 * sz)
constexpr int kPruneThreads = 512;          // two CTAs of 16 warps per SM

__global__ void __launch_bounds__(kPruneThreads) k_prune_tiled(const float2* __restrict__ fine, int N,
                                                    int npol, int beta, int sz, int R,
                                                    const float* __restrict__ z,
                                                    float2* __restrict__ pruned) {
    extern __shared__ __align__(16) float2 tilebuf[];      // [rows][kPruneCols], then Z
    const int hz = sz / 2, hb = beta / 2;
    const int c0 = blockIdx.x * kPruneCols;
    const int kstart = blockIdx.y * R;
    const int64_t fr = (int64_t)beta * N;
    const int C = N * npol;                                // fine-grid row length
    int64_t r_lo = (int64_t)(kstart - hz) * hb - beta / 4;
    int64_t r_hi = (int64_t)(kstart + R - 1 + hz) * hb - beta / 4 + hb;
    if (r_lo < 0) r_lo = 0;
    if (r_hi > fr) r_hi = fr;
    const int nrows = (int)(r_hi - r_lo);                  // <= kPruneRowsMax by the launch
    float* zs = reinterpret_cast<float*>(tilebuf + kPruneRowsMax * kPruneCols);
    for (int e = threadIdx.x; e < hb * sz; e += blockDim.x) zs[e] = z[e];
    for (int e = threadIdx.x; e < nrows * kPruneCols; e += blockDim.x) {
        const int rr = e / kPruneCols, cc = e - rr * kPruneCols;
        const int cg = c0 + cc;
        tilebuf[e] = cg < C ? fine[(r_lo + rr) * (int64_t)C + cg] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int c = threadIdx.x % kPruneCols;
    const int cg = c0 + c;
    const int u = cg / npol, p = cg - u * npol;
    for (int kk = threadIdx.x / kPruneCols; kk < R; kk += blockDim.x / kPruneCols) {
        const int k = kstart + kk;
        if (k >= 2 * N || cg >= C) continue;
        float ax = 0.f, ay = 0.f;
        for (int t = -hz; t <= hz; ++t) {
            const int64_t rs = (int64_t)(k - t) * hb - beta / 4;     // first row of k' = k - t
            const int m0 = rs < r_lo ? (int)(r_lo - rs) : 0;
            const int m1 = rs + hb > r_hi ? (int)(r_hi - rs) : hb;
            const float2* f = tilebuf + (rs - r_lo) * kPruneCols + c;
            const float* zt = zs + t + hz;
            for (int m = m0; m < m1; ++m) {
                const float wz = zt[m * sz];
                const float2 fv = f[m * kPruneCols];
                ax = fmaf(wz, fv.x, ax);
                ay = fmaf(wz, fv.y, ay);
            }
        }
        pruned[((int64_t)p * 2 * N + k) * N + u] = make_float2(ax, ay);
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

// Streaming pruner.  The pruning of one column is a polyphase filter: fine
// row r (2x row k' = nearest, offset m) feeds the S_z output rows
// k' - hz .. k' + hz.  A thread owns one fine-grid column (one polarisation
// of one u; a warp reads 32 contiguous ones) and a segment of output rows
// and walks the 2x rows k' in order: it reads the beta/2 fine rows of k'
// once (coalesced across the warp, streaming loads), adds them into a ring of
// S_z register accumulators and stores output row k' - hz, which no later k'
// touches.  The walk is unrolled by S_z from a multiple of S_z, so output k
// sits in accumulator k mod S_z at a compile-time index, and the Z weights
// are a by-value kernel argument, i.e. constant-bank operands of the FMAs.
// Each fine value is read from memory about once and there is no shared
// memory traffic: the kernel is bound by HBM bandwidth.
template <int HB, int SZ>
struct PruneZ {
    float z[HB * SZ];   // Z[m][t + hz]
};

template <int HB>
__device__ __forceinline__ void prune_rows(const float2* __restrict__ col, int64_t r0, int64_t fr,
                                           int64_t C, float2 (&f)[HB]) {
#pragma unroll
    for (int m = 0; m < HB; ++m) {
        const int64_t r = r0 + m;
        f[m] = (r >= 0 && r < fr) ? __ldcs(col + r * C) : make_float2(0.f, 0.f);
    }
}

template <int HB, int SZ>
__global__ void __launch_bounds__(256) k_prune_stream(const float2* __restrict__ fine, int N,
                                                      int npol, int L, const PruneZ<HB, SZ> Z,
                                                      float2* __restrict__ pruned) {
    constexpr int hz = SZ / 2;
    const int64_t C = (int64_t)N * npol;           // fine-grid row length (columns c = u npol + pol)
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int u = (int)(c / npol), p = (int)(c - (int64_t)u * npol);
    const int64_t fr = (int64_t)2 * HB * N;        // beta N fine rows
    const int rows2 = 2 * N;
    const float2* col = fine + c;
    float2* out = pruned + (int64_t)p * rows2 * N + u;
    const int kb = blockIdx.y * L;                 // this thread's output rows [kb, ke)
    const int ke = min(kb + L, rows2);
    if (kb >= ke) return;
    // 2x rows k' = kb - hz .. ke - 1 + hz, walked from a multiple of SZ
    const int a = kb - hz;
    const int g0 = a >= 0 ? a - a % SZ : -((-a + SZ - 1) / SZ) * SZ;
    const int glast = ke - 1 + hz;
    float2 acc[SZ];
#pragma unroll
    for (int q = 0; q < SZ; ++q) acc[q] = make_float2(0.f, 0.f);
    // fine rows of k' start at k' HB - beta / 4 = (k' - 1/2) HB; the rows of
    // the next PD 2x rows are in flight while k' is added (PD = 2 for
    // beta = 8, 1 for beta = 16 to bound the registers)
    constexpr int PD = HB == 4 ? 2 : 1;
    float2 fa[HB], fb[HB];
    prune_rows<HB>(col, (int64_t)g0 * HB - HB / 2, fr, C, fa);
    if (PD == 2) prune_rows<HB>(col, (int64_t)(g0 + 1) * HB - HB / 2, fr, C, fb);
    for (int g = g0; g <= glast; g += SZ) {
#pragma unroll
        for (int i = 0; i < SZ; ++i) {
            const int kp = g + i;
            float2 fc[HB];                          // PD 2x rows ahead
            prune_rows<HB>(col, (int64_t)(kp + PD) * HB - HB / 2, fr, C, fc);
#pragma unroll
            for (int t = -hz; t <= hz; ++t) {
                const int q = (i + t + SZ) % SZ;    // accumulator of output kp + t
#pragma unroll
                for (int m = 0; m < HB; ++m) {
                    const float w = Z.z[m * SZ + t + hz];
                    acc[q].x = fmaf(w, fa[m].x, acc[q].x);
                    acc[q].y = fmaf(w, fa[m].y, acc[q].y);
                }
            }
            const int k = kp - hz;                  // complete: no later k' reaches it
            const int qd = (i - hz + SZ) % SZ;
            if (k >= kb && k < ke) __stcs(out + (int64_t)k * N, acc[qd]);
            acc[qd] = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < HB; ++m) {
                if (PD == 2) {
                    fa[m] = fb[m];
                    fb[m] = fc[m];
                } else {
                    fa[m] = fc[m];
                }
            }
        }
    }
}

template <int HB, int SZ>
void launch_prune_stream(const float2* fine, int npol, int N, const float* h_z, int num_sms,
                         float2* pruned, cudaStream_t s) {
    PruneZ<HB, SZ> Z;
    for (int i = 0; i < HB * SZ; ++i) Z.z[i] = h_z[i];
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prune_stream<HB, SZ>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    // one wave: segments per column so that every resident thread owns one
    const int64_t resident = (int64_t)std::max(num_sms, 1) * per_sm * 256;
    const int64_t cols = (int64_t)npol * N;
    int64_t nseg = std::max<int64_t>(1, resident / cols);
    int64_t L = (2LL * N + nseg - 1) / nseg;
    if (L < SZ) L = SZ;
    nseg = (2LL * N + L - 1) / L;
    const dim3 grid((unsigned)((cols + 255) / 256), (unsigned)nseg, 1u);
    k_prune_stream<HB, SZ><<<grid, 256, 0, s>>>(fine, N, npol, (int)L, Z, pruned);
}

template <int HB>
bool launch_prune_stream_hb(const float2* fine, int npol, int N, int sz, const float* h_z,
                            int num_sms, float2* pruned, cudaStream_t s) {
    switch (sz) {
        case 7: launch_prune_stream<HB, 7>(fine, npol, N, h_z, num_sms, pruned, s); return true;
        case 9: launch_prune_stream<HB, 9>(fine, npol, N, h_z, num_sms, pruned, s); return true;
        case 11: launch_prune_stream<HB, 11>(fine, npol, N, h_z, num_sms, pruned, s); return true;
        case 13: launch_prune_stream<HB, 13>(fine, npol, N, h_z, num_sms, pruned, s); return true;
        case 15: launch_prune_stream<HB, 15>(fine, npol, N, h_z, num_sms, pruned, s); return true;
        default: return false;
    }
}

}  // namespace

void launch_hybrid_grid(const gw_index_rec* rec, int64_t nvis, const void* vis, int vis_kind,
                        const float* weight, int npol, int beta, int S, const double* c1,
                        int fmin, double norm, int N, int sz, float2* fine,
                        unsigned long long* dropped, cudaStream_t s) {
    if (nvis <= 0) return;
    const size_t tab = sizeof(float) * (size_t)beta * S;
    const int wtab = tab <= 16384 ? 1 : 0;
    const int G = S <= 32 ? 32 / S : 1;
    const int64_t warps = (nvis + G - 1) / G;
    k_hybrid_grid<<<blocks_for(warps * 32), 256, wtab ? tab : 0, s>>>(
        rec, nvis, vis, vis_kind, weight, npol, beta, S, c1, fmin, norm, N, sz, wtab, fine,
        dropped);
    note_launch();
}

void launch_prune(const float2* fine, int npol, int N, int beta, int sz, const float* z,
                  const float* h_z, int num_sms, float2* pruned, cudaStream_t s) {
    if (h_z) {
        const bool done = beta == 8 ? launch_prune_stream_hb<4>(fine, npol, N, sz, h_z, num_sms,
                                                                pruned, s)
                        : beta == 16 ? launch_prune_stream_hb<8>(fine, npol, N, sz, h_z, num_sms,
                                                                 pruned, s)
                                     : false;
        if (done) {
            note_launch();
            return;
        }
    }
    // largest power-of-two row block whose fine-row window fits the tile
    int R = 128;
    while (R >= 8 && ((int64_t)(R + sz) * beta / 2 + 2 > kPruneRowsMax)) R >>= 1;
    if (R >= 8 && (beta / 2) * sz <= kPruneZMax && npol <= 65535 &&
        (2LL * N + R - 1) / R <= 65535) {
        const size_t smem = sizeof(float2) * kPruneRowsMax * kPruneCols + sizeof(float) * kPruneZMax;
        cudaFuncSetAttribute(k_prune_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        const dim3 grid((unsigned)(((int64_t)N * npol + kPruneCols - 1) / kPruneCols),
                        (unsigned)((2LL * N + R - 1) / R), 1u);
        k_prune_tiled<<<grid, kPruneThreads, smem, s>>>(fine, N, npol, beta, sz, R, z, pruned);
    } else {
        k_prune<<<blocks_for((int64_t)npol * 2 * N * N), 256, 0, s>>>(fine, npol, N, beta, sz, z,
                                                                     pruned);
    }
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
