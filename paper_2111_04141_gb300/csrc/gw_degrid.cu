// Degridding kernel: the adjoint of gridding (operator G^T of Eq.
// (residualcalc), Section 1.6):
//     V[pol] = sum_{tv, tu} conj(K_i(tv, tu)) * G[pol][kv + tv][ku + tu],
// K_i the record's kernel (K_p[ov][ou], or its conjugate when w < 0).
// Tables of any storage kind are widened to FP32 on load, the sum is FP32,
// and the result is written in the plan's visibility kind.
//
// Two kernels:
// * k_degrid_staged (used by gw_degrid_vis): a CTA takes a work item of one
//   16 x 16 centre tile, copies the tile's grid region (the tile plus the
//   plan's largest half-support on every side, one plane per polarisation) into
//   shared memory once, and serves all records of the item from it, so the
//   grid is read from L2/HBM about once per tile instead of once per tap.
//   One warp per record: lanes take consecutive taps of the S x S footprint
//   (flattened, so every lane is busy), multiply-accumulate all polarisations
//   against the kernel slice (read coalesced from the table, one step ahead)
//   and reduce with warp shuffles.  The region fills most of an SM's shared
//   memory, so a CTA is 32 warps: the table loads from L2 are the latency to
//   hide, and planes per polarisation keep each lane's grid reads
//   conflict-light (8-byte stride).
// * k_degrid (the fallback when the region does not fit in shared memory,
//   and the allocation-free entry point): the same per-record warp, reading
//   the grid through L1/L2, records visited in 32 x 32 centre-tile order.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kThreads = 256;

template <int NPOL, int TK>
__global__ void __launch_bounds__(kThreads) k_degrid(DegridArgs a) {
    using TE = TabElem<TK>;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t n = *a.n_entries;
    const int N = a.N;
    const int hb = a.beta / 2;
    for (int64_t e = warp0; e < n; e += nwarps) {
        const uint32_t id = __ldg(a.entries + e);
        int4 rv = __ldg(reinterpret_cast<const int4*>(a.rec) + id);
        const gw_index_rec r = *reinterpret_cast<gw_index_rec*>(&rv);
        const int S = __ldg(a.support + r.plane), h = S >> 1;
        const typename TE::T* K = reinterpret_cast<const typename TE::T*>(a.table) +
                                  __ldg(a.plane_off + r.plane) +
                                  ((int64_t)(r.ov + hb) * a.beta + (r.ou + hb)) * S * S;
        // conj(K_i): K_i = K for w >= 0 (use conj K), K_i = conj K for w < 0 (use K)
        const float s = (r.flags & GW_FLAG_CONJ) ? -1.f : 1.f;
        float acc[NPOL][2];
#pragma unroll
        for (int p = 0; p < NPOL; ++p) acc[p][0] = acc[p][1] = 0.f;
        for (int tv = 0; tv < S; ++tv) {
            const int64_t row = r.kv - h + tv;
            for (int tu = lane; tu < S; tu += 32) {
                const float2 k = TE::load(K + tv * S + tu);
                const float ki = s * k.y;
                const int64_t col = r.ku - h + tu;
#pragma unroll
                for (int p = 0; p < NPOL; ++p) {
                    const float2 g = __ldg(a.grid + ((int64_t)p * N + row) * N + col);
                    // (k.x - j ki) * (g.x + j g.y)
                    acc[p][0] = fmaf(k.x, g.x, acc[p][0]);
                    acc[p][0] = fmaf(ki, g.y, acc[p][0]);
                    acc[p][1] = fmaf(k.x, g.y, acc[p][1]);
                    acc[p][1] = fmaf(-ki, g.x, acc[p][1]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < NPOL; ++p)
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                acc[p][0] += __shfl_xor_sync(0xffffffffu, acc[p][0], d);
                acc[p][1] += __shfl_xor_sync(0xffffffffu, acc[p][1], d);
            }
        if (lane < NPOL) {
            float re = acc[0][0], im = acc[0][1];
#pragma unroll
            for (int p = 1; p < NPOL; ++p)
                if (lane == p) { re = acc[p][0]; im = acc[p][1]; }
            store_vis(a.vis_out, a.vis_kind, (int64_t)id * NPOL + lane, re * a.table_inv,
                      im * a.table_inv);
        }
    }
}

template <int NPOL, int TK>
void launch_t(const DegridArgs& a, int64_t nvis, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid<NPOL, TK>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (nvis * 32 + kThreads - 1) / kThreads;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms * per_sm);
    if (blocks < 1) blocks = 1;
    k_degrid<NPOL, TK><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    note_launch();
}

constexpr int kStagedThreads = 1024;
constexpr int kStagedTile = 16;

template <int NPOL, int TK>
__global__ void __launch_bounds__(kStagedThreads) k_degrid_staged(DegridArgs a, int hmax) {
    using TE = TabElem<TK>;
    extern __shared__ __align__(16) float2 reg[];          // [NPOL][RS][RS]
    __shared__ uint32_t s_item;
    const int RS = kStagedTile + 2 * hmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = kStagedThreads / 32;
    const int N = a.N, hb = a.beta / 2;
    const uint32_t nitems = *a.item_count;
    for (;;) {
        __syncthreads();                       // previous item fully consumed
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= nitems) break;
        const Item item = a.items[it];
        const int rx0 = (item.tile % a.ntiles_u) * kStagedTile - hmax;
        const int ry0 = (item.tile / a.ntiles_u) * kStagedTile - hmax;
        // stage the region, polarisations interleaved
        for (int e = threadIdx.x; e < RS * RS; e += kStagedThreads) {
            const int y = e / RS, x = e - y * RS;
            const int gy = ry0 + y, gx = rx0 + x;
            const bool in = gx >= 0 && gx < N && gy >= 0 && gy < N;
#pragma unroll
            for (int p = 0; p < NPOL; ++p)
                reg[(size_t)p * RS * RS + e] =
                    in ? __ldg(a.grid + ((int64_t)p * N + gy) * N + gx) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int r = warp; r < item.len; r += nwarps) {
            const uint32_t id = __ldg(a.entries + item.start + r);
            int4 rv = __ldg(reinterpret_cast<const int4*>(a.rec) + id);
            const gw_index_rec rc = *reinterpret_cast<gw_index_rec*>(&rv);
            const int S = __ldg(a.support + rc.plane), h = S >> 1;
            const typename TE::T* K = reinterpret_cast<const typename TE::T*>(a.table) +
                                      __ldg(a.plane_off + rc.plane) +
                                      ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) * S * S;
            const float sg = (rc.flags & GW_FLAG_CONJ) ? -1.f : 1.f;
            // region index of tap (0, 0)
            const int base = (rc.kv - h - ry0) * RS + (rc.ku - h - rx0);
            float acc[NPOL][2];
#pragma unroll
            for (int p = 0; p < NPOL; ++p) acc[p][0] = acc[p][1] = 0.f;
            const int n = S * S;
            // flattened taps t = lane + 32 i, (tv, tu) advanced incrementally;
            // the kernel values of the next step load while this one's FMAs run
            const int dq = 32 / S, dr = 32 - dq * S;
            int tv = lane / S, tu = lane - (lane / S) * S;
            float2 k1 = lane < n ? TE::load(K + lane) : make_float2(0.f, 0.f);
            for (int t = lane; t < n; t += 32) {
                const float2 k = k1;
                if (t + 32 < n) k1 = TE::load(K + t + 32);
                const float ki = sg * k.y;
                const int off = base + tv * RS + tu;
#pragma unroll
                for (int p = 0; p < NPOL; ++p) {
                    const float2 gv = reg[(size_t)p * RS * RS + off];
                    // conj(K_i) G with K_i = K (w >= 0) or conj K (w < 0)
                    acc[p][0] = fmaf(k.x, gv.x, acc[p][0]);
                    acc[p][0] = fmaf(ki, gv.y, acc[p][0]);
                    acc[p][1] = fmaf(k.x, gv.y, acc[p][1]);
                    acc[p][1] = fmaf(-ki, gv.x, acc[p][1]);
                }
                tu += dr;
                tv += dq;
                if (tu >= S) {
                    tu -= S;
                    ++tv;
                }
            }
            if constexpr (NPOL == 4) {
                // reduce-scatter butterfly: lanes with bit 4 set keep pols 2, 3,
                // then bit 3 picks one of the two; 12 shuffles instead of 40
                const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
                const float k0r = (b4 ? acc[2][0] : acc[0][0]) +
                                  __shfl_xor_sync(0xffffffffu, b4 ? acc[0][0] : acc[2][0], 16);
                const float k0i = (b4 ? acc[2][1] : acc[0][1]) +
                                  __shfl_xor_sync(0xffffffffu, b4 ? acc[0][1] : acc[2][1], 16);
                const float k1r = (b4 ? acc[3][0] : acc[1][0]) +
                                  __shfl_xor_sync(0xffffffffu, b4 ? acc[1][0] : acc[3][0], 16);
                const float k1i = (b4 ? acc[3][1] : acc[1][1]) +
                                  __shfl_xor_sync(0xffffffffu, b4 ? acc[1][1] : acc[3][1], 16);
                float re = (b3 ? k1r : k0r) + __shfl_xor_sync(0xffffffffu, b3 ? k0r : k1r, 8);
                float im = (b3 ? k1i : k0i) + __shfl_xor_sync(0xffffffffu, b3 ? k0i : k1i, 8);
#pragma unroll
                for (int d = 4; d > 0; d >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, d);
                    im += __shfl_xor_sync(0xffffffffu, im, d);
                }
                if ((lane & 7) == 0) {
                    const int p = (b4 ? 2 : 0) + (b3 ? 1 : 0);
                    store_vis(a.vis_out, a.vis_kind, (int64_t)id * NPOL + p, re * a.table_inv,
                              im * a.table_inv);
                }
            } else {
#pragma unroll
                for (int p = 0; p < NPOL; ++p)
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) {
                        acc[p][0] += __shfl_xor_sync(0xffffffffu, acc[p][0], d);
                        acc[p][1] += __shfl_xor_sync(0xffffffffu, acc[p][1], d);
                    }
                if (lane < NPOL) {
                    float re = acc[0][0], im = acc[0][1];
#pragma unroll
                    for (int p = 1; p < NPOL; ++p)
                        if (lane == p) { re = acc[p][0]; im = acc[p][1]; }
                    store_vis(a.vis_out, a.vis_kind, (int64_t)id * NPOL + lane, re * a.table_inv,
                              im * a.table_inv);
                }
            }
        }
    }
}

template <int NPOL, int TK>
bool launch_staged_t(const DegridArgs& a, int hmax, int num_sms, cudaStream_t s) {
    const int RS = kStagedTile + 2 * hmax;
    const size_t smem = (size_t)RS * RS * NPOL * sizeof(float2);
    if (smem > kStagedSmemMax) return false;
    cudaFuncSetAttribute(k_degrid_staged<NPOL, TK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid_staged<NPOL, TK>,
                                                  kStagedThreads, smem);
    if (per_sm < 1) return false;
    k_degrid_staged<NPOL, TK><<<num_sms * per_sm, kStagedThreads, smem, s>>>(a, hmax);
    note_launch();
    return true;
}

template <int TK>
bool launch_staged_k(const DegridArgs& a, int hmax, int num_sms, cudaStream_t s) {
    switch (a.npol) {
        case 1: return launch_staged_t<1, TK>(a, hmax, num_sms, s);
        case 2: return launch_staged_t<2, TK>(a, hmax, num_sms, s);
        case 3: return launch_staged_t<3, TK>(a, hmax, num_sms, s);
        default: return launch_staged_t<4, TK>(a, hmax, num_sms, s);
    }
}

template <int TK>
void launch_k(const DegridArgs& a, int64_t nvis, int num_sms, cudaStream_t s) {
    switch (a.npol) {
        case 1: launch_t<1, TK>(a, nvis, num_sms, s); break;
        case 2: launch_t<2, TK>(a, nvis, num_sms, s); break;
        case 3: launch_t<3, TK>(a, nvis, num_sms, s); break;
        default: launch_t<4, TK>(a, nvis, num_sms, s); break;
    }
}

}  // namespace

int degrid_staged_tile() { return kStagedTile; }

cudaError_t preload_degrid_kernel(int npol, int table_kind) {
    cudaFuncAttributes attr;
    auto get = [&](auto f) { return cudaFuncGetAttributes(&attr, f); };
    const int tk = table_kind == GW_BF16X2 ? 1 : (table_kind == GW_F16X2 ? 2 : 0);
    switch (npol * 3 + tk) {
        case 3: return get(k_degrid<1, GW_C64>);
        case 4: return get(k_degrid<1, GW_BF16X2>);
        case 5: return get(k_degrid<1, GW_F16X2>);
        case 6: return get(k_degrid<2, GW_C64>);
        case 7: return get(k_degrid<2, GW_BF16X2>);
        case 8: return get(k_degrid<2, GW_F16X2>);
        case 9: return get(k_degrid<3, GW_C64>);
        case 10: return get(k_degrid<3, GW_BF16X2>);
        case 11: return get(k_degrid<3, GW_F16X2>);
        case 13: return get(k_degrid<4, GW_BF16X2>);
        case 14: return get(k_degrid<4, GW_F16X2>);
        default: return get(k_degrid<4, GW_C64>);
    }
}

bool degrid_staged_fits(int hmax, int npol) {
    const int RS = kStagedTile + 2 * hmax;
    return (size_t)RS * RS * npol * sizeof(float2) <= kStagedSmemMax;
}

bool launch_degrid_staged(const DegridArgs& a, int hmax, int num_sms, cudaStream_t s) {
    cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
    switch (a.table_kind) {
        case GW_BF16X2: return launch_staged_k<GW_BF16X2>(a, hmax, num_sms, s);
        case GW_F16X2: return launch_staged_k<GW_F16X2>(a, hmax, num_sms, s);
        default: return launch_staged_k<GW_C64>(a, hmax, num_sms, s);
    }
}

void launch_degrid(const DegridArgs& a, int64_t nvis, int num_sms, cudaStream_t s) {
    switch (a.table_kind) {
        case GW_BF16X2: launch_k<GW_BF16X2>(a, nvis, num_sms, s); break;
        case GW_F16X2: launch_k<GW_F16X2>(a, nvis, num_sms, s); break;
        default: launch_k<GW_C64>(a, nvis, num_sms, s); break;
    }
}

}  // namespace gw
