// Degridding kernel: the adjoint of gridding (operator G^T of Eq.
// (residualcalc), Section 1.6):
//     V[pol] = sum_{tv, tu} conj(K_i(tv, tu)) * G[pol][kv + tv][ku + tu],
// K_i the record's kernel (K_p[ov][ou], or its conjugate when w < 0).
// Tables of any storage kind are widened to FP32 on load, the sum is FP32,
// and the result is written in the plan's visibility kind.
//
// Two kernels:
// * k_degrid_staged (used by gw_degrid_vis): one CTA of 24 warps per SM
//   serves chunks of work items (at most 1,024 records centred in one 16 x 16
//   tile).  Warps 0-3 load the records' metadata (id, kernel slice, centre,
//   support) into one of two shared buffers, the next chunk's while all
//   warps compute the current one.  The CTA stages the tile's grid region
//   (the tile plus the chunk's largest half-support on every side) in
//   shared memory once, as polarisation pairs, at a row pitch padded to the
//   support residue (mod 8) that carries most of the item's taps, and serves
//   all of the item's records from it, so the grid is read from L2/HBM
//   about once per tile instead of once per tap.  Warps claim records one at
//   a time, wide supports first.  One warp per record: lanes take
//   consecutive taps of the S x S footprint (flattened, so every lane is
//   busy), with kernel values loaded four steps ahead, packed FP32x2 FMAs
//   into K.re G and K.im G sums, and a reduce-scatter over the lanes.
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

#ifndef GW_DEGRID_THREADS
#define GW_DEGRID_THREADS 768
#endif
constexpr int kStagedThreads = GW_DEGRID_THREADS;
constexpr int kStagedTile = 16;
constexpr int kStagedMeta = 1024;   // records whose metadata a CTA stages at once
constexpr int kStagedPad = 4;       // zero elements after each staged plane
#ifndef GW_DEGRID_DEPTH
#define GW_DEGRID_DEPTH 4
#endif
constexpr int kStagedDepth = GW_DEGRID_DEPTH;   // steps of kernel values loaded ahead

// A chunk: at most kStagedMeta records of a work item (items longer than
// that are served in several chunks from one staged region), with its record
// metadata in one of two shared buffers.
struct StagedChunk {
    Item item;
    int c0, nc;     // first record of the chunk in the item, records in it
    int done;       // no work left
    int h;          // largest half-support of the chunk's records (the region's)
    int front, back, next;   // metadata placement, record claims
    int taps[8];    // taps of the chunk's records by S mod 8
};

constexpr int kLoaderThreads = 128;                       // warps 0-3
constexpr int kMetaPerLoader = kStagedMeta / kLoaderThreads;
constexpr int kLoaderBatch = 4;                           // records whose loads a loader issues together

__device__ __forceinline__ void loader_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
}

template <int NPOL, int TK>
__global__ void __launch_bounds__(kStagedThreads) k_degrid_staged(DegridArgs a, int hmax) {
    using TE = TabElem<TK>;
    using T = typename TE::T;
    constexpr int D = kStagedDepth;
    // grid region as polarisation pairs [NPOL / 2][RS][RS] of (G_p, G_p+1),
    // then [RS][RS] of the last polarisation if NPOL is odd; two chunks'
    // record metadata after the largest region (RS = 16 + 2 h_max)
    constexpr int NPR = NPOL / 2;
    extern __shared__ __align__(16) float4 reg[];
    __shared__ StagedChunk s_ch[2];
    uint4* meta0;
    {
        const int RSM = kStagedTile + 2 * hmax, pm = RSM * RSM + kStagedPad;
        meta0 = reinterpret_cast<uint4*>(reinterpret_cast<float2*>(reg + (size_t)NPR * pm) +
                                         (NPOL % 2 ? pm : 0));
    }
    const int lane = threadIdx.x & 31;
    const int N = a.N, hb = a.beta / 2;
    const uint32_t nitems = *a.item_count;
    const T* __restrict__ tab = reinterpret_cast<const T*>(a.table);
    // thread 0: the item being served and the next chunk's first record
    Item cur{};
    int next_c0 = 0;

    // The loader warps (0-3) pick the next chunk and load its records'
    // metadata (id, kernel slice offset, centre relative to the tile,
    // support | conj << 16) into buffer `buf`, records wider than h_max / 2
    // first: warps claim records in this order, so the long ones start early
    // and the short ones even out the end of the chunk.  Each loader thread
    // issues the loads of its (up to 8) records together.
    auto load_chunk = [&](const int buf) {
        StagedChunk& c = s_ch[buf];
        if (threadIdx.x == 0) {
            c.done = 0;
            if (next_c0 == 0 || next_c0 >= cur.len) {
                const uint32_t it = atomicAdd(a.queue, 1u);
                c.done = it >= nitems;
                if (it < nitems) cur = a.items[it];
                next_c0 = 0;
            }
            const int nc = min(kStagedMeta, cur.len - next_c0);
            c.item = cur;
            c.c0 = next_c0;
            c.nc = nc;
            c.next = 0;
            c.front = 0;
            c.back = nc;
            // an item served in several chunks keeps one region for all of
            // them: the plan's largest half-support
            c.h = cur.len > kStagedMeta ? hmax : 0;
            for (int k = 0; k < 8; ++k) c.taps[k] = 0;
            next_c0 += nc;
        }
        loader_sync();
        if (c.done) return;
        const Item item = c.item;
        const int c0 = c.c0, nc = c.nc;
        const int tx0 = (item.tile % a.ntiles_u) * kStagedTile;
        const int ty0 = (item.tile / a.ntiles_u) * kStagedTile;
        uint4* meta = meta0 + buf * kStagedMeta;
        int hw = 0;
        for (int k0 = 0; k0 < kMetaPerLoader; k0 += kLoaderBatch) {
            uint32_t ids[kLoaderBatch];
            gw_index_rec rcs[kLoaderBatch];
#pragma unroll
            for (int k = 0; k < kLoaderBatch; ++k) {
                const int r = (k0 + k) * kLoaderThreads + threadIdx.x;
                ids[k] = r < nc ? __ldg(a.entries + item.start + c0 + r) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kLoaderBatch; ++k) {
                const int r = (k0 + k) * kLoaderThreads + threadIdx.x;
                if (r < nc) {
                    int4 rv = __ldg(reinterpret_cast<const int4*>(a.rec) + ids[k]);
                    rcs[k] = *reinterpret_cast<gw_index_rec*>(&rv);
                }
            }
#pragma unroll
            for (int k = 0; k < kLoaderBatch; ++k) {
                const int r = (k0 + k) * kLoaderThreads + threadIdx.x;
                if (r < nc) {
                    const gw_index_rec rc = rcs[k];
                    const int S = __ldg(a.support + rc.plane), h = S >> 1;
                    const int64_t kofs = __ldg(a.plane_off + rc.plane) +
                                         ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) * S * S;
                    uint32_t rel = (uint32_t)(rc.ku - tx0) | (uint32_t)(rc.kv - ty0) << 8;
                    uint32_t w = (uint32_t)S | ((rc.flags & GW_FLAG_CONJ) ? 1u << 16 : 0u);
#ifdef GW_DEBUG_BOUNDS
                    // the record's slice, centre tile, region and output row: a
                    // record that fails is replaced by a 1 x 1 one at the
                    // table's start, centred in the tile
                    const bool ok =
                        (a.table_elems == 0 || (kofs >= 0 && kofs + (int64_t)S * S <= a.table_elems)) &&
                        rc.ku - tx0 >= 0 && rc.ku - tx0 < kStagedTile && rc.kv - ty0 >= 0 &&
                        rc.kv - ty0 < kStagedTile && h <= hmax &&
                        (a.vis_count == 0 || ids[k] < (uint64_t)a.vis_count);
                    if (!gw_in_bounds(ok, a.queue + 1)) {
                        rel = 8u | 8u << 8;
                        w = 1u;
                    }
#endif
                    const int pos =
                        h > hmax / 2 ? atomicAdd(&c.front, 1) : atomicSub(&c.back, 1) - 1;
#ifdef GW_DEBUG_BOUNDS
                    if (!gw_in_bounds(pos >= 0 && pos < nc, a.queue + 1)) continue;
                    if ((w & 0xffffu) == 1u && S != 1) {
                        meta[pos] = make_uint4(0u, 0u, rel, w);
                        continue;
                    }
#endif
                    meta[pos] = make_uint4(ids[k], (uint32_t)kofs, rel, w);
                    hw = max(hw, h);
                    atomicAdd(&c.taps[S & 7], S * S);
                }
            }
            if ((k0 + kLoaderBatch) * kLoaderThreads >= nc) break;
        }
        hw = (int)__reduce_max_sync(0xffffffffu, (unsigned)hw);
        if (lane == 0 && hw > 0) atomicMax(&c.h, hw);
    };

    if (threadIdx.x < kLoaderThreads) load_chunk(0);
    __syncthreads();
    for (int kc = 0;; ++kc) {
        const int buf = kc & 1;
        const StagedChunk& c = s_ch[buf];
        if (c.done) break;
        const Item item = c.item;
        const int c0 = c.c0, nc = c.nc;
        const int tx0 = (item.tile % a.ntiles_u) * kStagedTile;
        const int ty0 = (item.tile / a.ntiles_u) * kStagedTile;
        const uint4* meta = meta0 + buf * kStagedMeta;
        // the region: rows and columns [t0 - hi, t0 + 16 + hi) of the tile,
        // RS x RS values at row pitch RSP; each plane holds RS x RSP elements
        // and kStagedPad zeros (element RS * RSP is read by lanes without a
        // tap in a record's last step).  A quarter-warp's 8 flattened taps
        // that cross a footprint row end jump by RSP - S elements: with RSP
        // = S mod 8 its 16-byte loads stay free of bank conflicts, so the
        // pitch is padded to the residue of the supports that carry most of
        // the item's taps, where the shared memory allows (items served in
        // several chunks keep RSP = RS).  RS is even, so every part stays
        // 16-byte aligned.
        const int hi = c.h;
        const int RS = kStagedTile + 2 * hi;
        int RSP = RS;
        if (item.len <= kStagedMeta) {
            int best = 0, bt = -1;
#pragma unroll
            for (int k = 1; k < 8; k += 2)     // supports are odd
                if (c.taps[k] > bt) {
                    bt = c.taps[k];
                    best = k;
                }
            const int rsp = RS + ((best - RS) & 7);
            const int RSM = kStagedTile + 2 * hmax;
            if (RS * rsp <= RSM * RSM) RSP = rsp;
        }
        const int plane = RS * RSP + kStagedPad;
        const int zoff = RS * RSP;
        float2* single = reinterpret_cast<float2*>(reg + (size_t)NPR * plane);
        if (c0 == 0) {
            const int rx0 = tx0 - hi, ry0 = ty0 - hi;
            if (threadIdx.x < kStagedPad) {
#pragma unroll
                for (int q = 0; q < NPR; ++q)
                    reg[(size_t)q * plane + zoff + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (NPOL % 2) single[zoff + threadIdx.x] = make_float2(0.f, 0.f);
            }
            for (int e0 = threadIdx.x; e0 < RS * RS; e0 += kStagedThreads) {
                const int y = e0 / RS, x = e0 - y * RS;
                const int e = y * RSP + x;
                const int gy = ry0 + y, gx = rx0 + x;
                const bool in = gx >= 0 && gx < N && gy >= 0 && gy < N;
                float2 g[NPOL];
#pragma unroll
                for (int p = 0; p < NPOL; ++p)
                    g[p] = in ? __ldg(a.grid + ((int64_t)p * N + gy) * N + gx) : make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < NPR; ++q)
                    reg[(size_t)q * plane + e] = make_float4(g[2 * q].x, g[2 * q].y, g[2 * q + 1].x,
                                                             g[2 * q + 1].y);
                if (NPOL % 2) single[e] = g[NPOL - 1];
            }
            __syncthreads();
        }
        // the loaders prepare the next chunk, then join the record claims
        if (threadIdx.x < kLoaderThreads) load_chunk(buf ^ 1);
        for (;;) {
            int r = 0;
            if (lane == 0) r = atomicAdd(&s_ch[buf].next, 1);
            r = __shfl_sync(0xffffffffu, r, 0);
            if (r >= nc) break;
            const uint4 m = meta[r];
            const uint32_t id = m.x;
            const T* K = tab + m.y;
            const int S = (int)(m.w & 0xffffu);
            const float sg = (m.w >> 16) ? -1.f : 1.f;
            const int n = S * S;
            // flattened taps t = lane + 32 i; the region index advances by
            // `step` per 32 taps, plus `wrap` when the tap column wraps
            const int dq = 32 / S, dr = 32 - dq * S;
            const int step = dq * RSP + dr, wrap = RSP - S;
            int tu = lane % S;
            // region index of tap (0, 0): centre - h + hi on both axes
            const int base = ((int)(m.z >> 8) - (S >> 1) + hi) * RSP + ((int)(m.z & 0xffu) - (S >> 1) + hi);
            int off = base + (lane / S) * RSP + tu;
            // a1 = sum K.re G, a2 = sum K.im G (packed FP32x2 FMAs); the
            // conjugation sign is applied once at the end
            float2 a1[NPOL], a2[NPOL];
#pragma unroll
            for (int p = 0; p < NPOL; ++p) a1[p] = a2[p] = make_float2(0.f, 0.f);
            auto tap = [&](const float2 k, const int o) {
                const float2 kxx = make_float2(k.x, k.x), kyy = make_float2(k.y, k.y);
#pragma unroll
                for (int q = 0; q < NPR; ++q) {
                    const float4 g = reg[(size_t)q * plane + o];
                    const float2 g0 = make_float2(g.x, g.y), g1 = make_float2(g.z, g.w);
                    a1[2 * q] = __ffma2_rn(kxx, g0, a1[2 * q]);
                    a2[2 * q] = __ffma2_rn(kyy, g0, a2[2 * q]);
                    a1[2 * q + 1] = __ffma2_rn(kxx, g1, a1[2 * q + 1]);
                    a2[2 * q + 1] = __ffma2_rn(kyy, g1, a2[2 * q + 1]);
                }
                if (NPOL % 2) {
                    const float2 g = single[o];
                    a1[NPOL - 1] = __ffma2_rn(kxx, g, a1[NPOL - 1]);
                    a2[NPOL - 1] = __ffma2_rn(kyy, g, a2[NPOL - 1]);
                }
            };
            auto advance = [&]() {
                off += step;
                tu += dr;
                if (tu >= S) {
                    tu -= S;
                    off += wrap;
                }
            };
            // steps 0 .. nfull - 1 have a tap on every lane, step nfull on
            // the lanes below n - 32 nfull.  Kernel values are loaded D steps
            // ahead, unconditionally: past the slice they read the next
            // slice or the table's zero slack, never used.
            const int nfull = (n - 1) >> 5;
            const T* kp = K + lane;
            T kq[D];
#pragma unroll
            for (int d = 0; d < D; ++d) kq[d] = __ldg(kp + 32 * d);
            kp += 32 * D;
            int i = 0;
            for (; i + D <= nfull; i += D) {
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float2 k = TE::cvt(kq[d]);
                    kq[d] = __ldg(kp + 32 * d);
                    tap(k, off);
                    advance();
                }
                kp += 32 * D;
            }
            // the last (< D) full steps and the partial one, from the front
            // of the ring
            for (; i <= nfull; ++i) {
                const bool live = i < nfull || lane + 32 * nfull < n;
                tap(live ? TE::cvt(kq[0]) : make_float2(0.f, 0.f), live ? off : zoff);
                advance();
#pragma unroll
                for (int d = 0; d + 1 < D; ++d) kq[d] = kq[d + 1];
            }
            // conj(K_i) G with K_i = K (w >= 0) or conj K (w < 0):
            // re = sum K.re G.re + s K.im G.im, im = sum K.re G.im - s K.im G.re
            float acc[NPOL][2];
#pragma unroll
            for (int p = 0; p < NPOL; ++p) {
                acc[p][0] = fmaf(sg, a2[p].y, a1[p].x);
                acc[p][1] = fmaf(-sg, a2[p].x, a1[p].y);
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
        __syncthreads();   // chunk consumed, the next chunk's metadata in place
    }
}

template <int NPOL, int TK>
bool launch_staged_t(const DegridArgs& a, int hmax, int num_sms, cudaStream_t s) {
    const int RS = kStagedTile + 2 * hmax;
    if ((size_t)RS * RS * NPOL * sizeof(float2) > kStagedSmemMax) return false;
    const size_t smem = (size_t)(RS * RS + kStagedPad) * NPOL * sizeof(float2) +
                        2 * kStagedMeta * sizeof(uint4);
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
