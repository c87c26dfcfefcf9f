// Gridding kernel: w-projection convolutional gridding onto a complex grid.
//
// Computes the Gridding Step of Algorithm convgriddingoversampling
// (Section 2.4.5) with the w-projection GCF (Section 1.7.1):
//     G[pol][kv + tv][ku + tu] += K_p[ov][ou](tv, tu) * V[pol]   (conj K if w < 0)
//
// Design (GB300): each CTA owns one kTile x kTile tile of the grid for the
// whole of a work item (a run of that tile's bin) and keeps the tile's
// accumulators in registers, so every grid point is read-modify-written once
// per work item instead of once per visibility.  A warp owns an 8 x 16
// block of the tile: lane (lu, lv) holds the points (lu, lv + 4 j), j = 0..3,
// for all polarisations.  Visibilities are staged in shared memory in
// batches; for each one a warp skips it unless the footprint meets its
// block, and skips each 8 x 4 slot the footprint's rows miss, so the
// granularity of wasted multiply-adds is an 8 x 4 patch.  Kernel values come
// through the read-only cache (the tables stay resident in L2).  Per tap and
// polarisation the update is 4 FFMA:
//     acc.re += K.re A.re + K.im B.re,  acc.im += K.re A.im + K.im B.im
// with A = V and B = (-V.im, V.re) (or (V.im, -V.re) for the conjugate
// kernel), precomputed per visibility, so conjugation costs nothing per tap.
// Work items of one tile commit with vector atomics (red.global.add); CTAs
// are persistent and pull items from a queue.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 256;

__device__ __forceinline__ gw_index_rec load_rec(const gw_index_rec* rec, uint32_t i) {
    int4 v = __ldg(reinterpret_cast<const int4*>(rec) + i);
    return *reinterpret_cast<gw_index_rec*>(&v);
}

template <int NPOL>
__global__ void __launch_bounds__(kThreads) k_grid(GridArgs a) {
    __shared__ int4 s_idx[kBatch];
    __shared__ float4 s_v[kBatch][NPOL];
    __shared__ uint32_t s_item;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bu = (warp & 3) * 8, bv = (warp >> 2) * 16;
    const int lu = lane & 7, lv = lane >> 3;
    const uint32_t nitems = *a.item_count;
    const int N = a.N;
    const int hb = a.beta / 2;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const Item item = a.items[it];
        const int tu0 = (item.tile % a.ntiles_side) * kTile;
        const int tv0 = (item.tile / a.ntiles_side) * kTile;

        float acc[4][NPOL][2];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int p = 0; p < NPOL; ++p) acc[j][p][0] = acc[j][p][1] = 0.f;

        for (int b0 = 0; b0 < item.len; b0 += kBatch) {
            const int nb = min(kBatch, item.len - b0);
            if ((int)threadIdx.x < nb) {
                const uint32_t id = __ldg(a.entries + item.start + b0 + threadIdx.x);
                const gw_index_rec r = load_rec(a.rec, id);
                const int S = __ldg(a.support + r.plane);
                const int64_t off = __ldg(a.plane_off + r.plane) +
                                    ((int64_t)(r.ov + hb) * a.beta + (r.ou + hb)) * S * S;
                s_idx[threadIdx.x] = make_int4(r.ku, r.kv, S, (int)off);
                const bool conj = (r.flags & GW_FLAG_CONJ) != 0;
#pragma unroll
                for (int p = 0; p < NPOL; ++p) {
                    float2 v = __ldg(a.vis + (int64_t)id * NPOL + p);
                    if (a.weight) {
                        const float w = __ldg(a.weight + (int64_t)id * NPOL + p);
                        v.x *= w;
                        v.y *= w;
                    }
                    s_v[threadIdx.x][p] = conj ? make_float4(v.x, v.y, v.y, -v.x)
                                               : make_float4(v.x, v.y, -v.y, v.x);
                }
            }
            __syncthreads();
            for (int r = 0; r < nb; ++r) {
                const int4 ri = s_idx[r];
                const int S = ri.z, h = S >> 1;
                const int du0 = tu0 + bu - ri.x;
                if (du0 + 7 < -h || du0 > h) continue;
                const int dv0 = tv0 + bv - ri.y;
                if (dv0 + 15 < -h || dv0 > h) continue;
                const int tu = du0 + lu;
                const bool oku = (tu >= -h) && (tu <= h);
                float4 V[NPOL];
#pragma unroll
                for (int p = 0; p < NPOL; ++p) V[p] = s_v[r][p];
                const float2* krow = a.table + ri.w + (tu + h);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int dvj = dv0 + 4 * j;
                    if (dvj + 3 < -h || dvj > h) continue;
                    const int tv = dvj + lv;
                    float2 K = make_float2(0.f, 0.f);
                    if (oku && tv >= -h && tv <= h) K = __ldg(krow + (tv + h) * S);
#pragma unroll
                    for (int p = 0; p < NPOL; ++p) {
                        acc[j][p][0] = fmaf(K.x, V[p].x, acc[j][p][0]);
                        acc[j][p][0] = fmaf(K.y, V[p].z, acc[j][p][0]);
                        acc[j][p][1] = fmaf(K.x, V[p].y, acc[j][p][1]);
                        acc[j][p][1] = fmaf(K.y, V[p].w, acc[j][p][1]);
                    }
                }
            }
            __syncthreads();
        }
        // commit the tile
        const int u = tu0 + bu + lu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int v = tv0 + bv + 4 * j + lv;
            if (u >= N || v >= N) continue;
#pragma unroll
            for (int p = 0; p < NPOL; ++p) {
                if (acc[j][p][0] != 0.f || acc[j][p][1] != 0.f)
                    atomicAdd(a.grid + ((int64_t)p * N + v) * N + u,
                              make_float2(acc[j][p][0], acc[j][p][1]));
            }
        }
    }
}

template <int NPOL>
void launch_t(const GridArgs& a, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid<NPOL>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    k_grid<NPOL><<<num_sms * per_sm, kThreads, 0, s>>>(a);
    note_launch();
}

}  // namespace

void launch_grid(const GridArgs& a, int num_sms, cudaStream_t s) {
    cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
    switch (a.npol) {
        case 1: launch_t<1>(a, num_sms, s); break;
        case 2: launch_t<2>(a, num_sms, s); break;
        case 3: launch_t<3>(a, num_sms, s); break;
        default: launch_t<4>(a, num_sms, s); break;
    }
}

}  // namespace gw
