// Gridding kernel: w-projection convolutional gridding onto a complex grid.
//
// Computes the Gridding Step of Algorithm convgriddingoversampling
// (Section 2.4.5) with the w-projection GCF (Section 1.7.1):
//     G[pol][kv + tv][ku + tu] += K_p[ov][ou](tv, tu) * V[pol]   (conj K if w < 0)
//
// Design (GB300):
// * A CTA owns one 32 (u) x 16 (v) tile of the grid for a work item (a run of
//   that tile's bin).  Sixteen consumer warps each own one 8 x 4 block of the
//   tile (lane (lu, lv) holds point (lu, lv) for every polarisation) and keep
//   its accumulators in registers for the whole work item, so each grid point
//   is committed once per work item (vector atomics, red.global).
// * A warpgroup of four producer warps walks the work item in batches and
//   appends, for every record, one 8-byte entry (table index of the tile
//   origin relative to the record, visibility id, conjugation bit) to the
//   list of every consumer warp whose block the record's footprint meets
//   (warp-aggregated shared atomics; four batches in flight, handed over with
//   named barriers).  A consumer reads one entry per record that touches its
//   block and runs no other per-record control: wasted multiply-adds are
//   limited to the parts of an 8 x 4 block outside a footprint.
// * Kernel values come from zero-padded slices (7 zero columns and 3 zero
//   rows around each S x S slice, one compile-time row stride per plan), so
//   lanes outside the footprint read zeros without predication.  Visibilities
//   are read straight from the visibility array with broadcast loads (the
//   shared-memory path is the scarce one).  Kernel values and visibilities of
//   the next two entries are in flight while one entry's multiply-adds issue.
// * Per tap and polarisation the complex update costs two packed FP32x2 FMAs
//   (Blackwell FFMA2: two multiply-adds per issued instruction), accumulated
//   as P = sum K (.) V and Q = sum (K.y, K.x) (.) V, separately for records
//   that use the kernel and for those that use its conjugate (w < 0); the
//   real and imaginary parts are formed at commit.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kColBlocks = 4, kRowBlocks = 4;            // 8 x 4 blocks per tile
constexpr int kComputeWarps = kColBlocks * kRowBlocks;   // one 8 x 4 block per warp
constexpr int kThreads = (kComputeWarps + 4) * 32;       // + one producer warpgroup
constexpr int kSyncThreads = kThreads;                   // threads in the batch barriers
constexpr int kProducerThreads = 4 * 32;                 // producer-only barrier (id 9)
constexpr int kBatch = 256;
constexpr int kBufs = 4;             // batches in flight (barriers 1..4 full, 5..8 empty)
constexpr int kTileU = 8 * kColBlocks, kTileV = 4 * kRowBlocks;
static_assert(kTileU == kGridTileU && kTileV == kGridTileV, "tile shape");

__device__ __forceinline__ gw_index_rec load_rec(const gw_index_rec* rec, uint32_t i) {
    int4 v = __ldg(reinterpret_cast<const int4*>(rec) + i);
    return *reinterpret_cast<gw_index_rec*>(&v);
}

__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <int NPOL>
struct Smem {
    // per consumer warp: (padded-table index of the tile origin for the record,
    // visibility id | conj << 31) of every record meeting the warp's block
    int2 list[kBufs][kComputeWarps][kBatch];
    int cnt[kBufs][kComputeWarps];
    int tile[kBufs];                       // tile of the batch; -1 = end of work
    int last[kBufs];                       // batch ends its work item
    uint32_t item;                         // work item fetched by the first producer warp
};

template <int NPOL, int SP>
__global__ void __launch_bounds__(kThreads, 1) k_grid(GridArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<NPOL>& sm = *reinterpret_cast<Smem<NPOL>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int side_u = a.ntiles_u;
    const int hb = a.beta / 2;

    if (warp >= kComputeWarps) {
        // ------------------------------------------------------------ producers
        // The four warps of this warpgroup stage each batch together: warp pw
        // takes records pw, pw + 4, ... of every 128-record group.
        const int pw = warp - kComputeWarps;
        const uint32_t nitems = *a.item_count;
        int buf = 0, uses = 0;
        for (;;) {
            if (warp == kComputeWarps && lane == 0) sm.item = atomicAdd(a.queue, 1u);
            bar_sync(9, kProducerThreads);
            const uint32_t it = sm.item;
            bar_sync(9, kProducerThreads);   // everyone has read sm.item
            const bool done = it >= nitems;
            Item item{};
            if (!done) item = a.items[it];
            const int nb_total = done ? 1 : (item.len + kBatch - 1) / kBatch;
            for (int b = 0; b < nb_total; ++b) {
                if (uses >= kBufs) bar_sync(1 + kBufs + buf, kSyncThreads);  // wait until consumed
                if (pw == 0 && lane < kComputeWarps) sm.cnt[buf][lane] = 0;
                bar_sync(9, kProducerThreads);   // counters cleared before any append
                if (done) {
                    if (pw == 0 && lane == 0) {
                        sm.tile[buf] = -1;
                        sm.last[buf] = 1;
                    }
                } else {
                    const int tu0 = (item.tile % side_u) * kTileU;
                    const int tv0 = (item.tile / side_u) * kTileV;
                    const int b0 = b * kBatch;
                    const int nb = min(kBatch, item.len - b0);
                    for (int g = 0; g < nb; g += 128) {
                        const int r = g + lane * 4 + pw;
                        const bool act = r < nb;
                        int base = 0;
                        uint32_t vidc = 0;
                        int cu0 = 1, cu1 = 0, cv0 = 1, cv1 = 0, vlo = 0, vhi = -1;
                        if (act) {
                            const uint32_t id = __ldg(a.entries + item.start + b0 + r);
                            const gw_index_rec rc = load_rec(a.rec, id);
                            const int S = __ldg(a.support + rc.plane), h = S >> 1;
                            const int64_t slice = __ldg(a.pplane_off + rc.plane) +
                                                  ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) *
                                                      (int64_t)(S + 6) * SP;
                            // padded index of the tile origin relative to this record
                            base = (int)slice + (tv0 - rc.kv + h + 3) * SP + (tu0 - rc.ku + h + 7);
                            vidc = id | ((rc.flags & GW_FLAG_CONJ) ? 0x80000000u : 0u);
                            // footprint relative to the tile
                            const int ulo = rc.ku - h - tu0, uhi = rc.ku + h - tu0;
                            vlo = rc.kv - h - tv0;
                            vhi = rc.kv + h - tv0;
                            cu0 = max(0, ulo) >> 3;
                            cu1 = min(kTileU - 1, uhi) >> 3;
                            cv0 = 0;
                            cv1 = (vhi >= 0 && vlo <= kTileV - 1) ? 0 : -1;
                        }
                        // warp-aggregated appends: one shared atomic per target warp
                        const int j0 = max(0, vlo) >> 2, j1 = min(kTileV - 1, vhi) >> 2;
                        for (int w = 0; w < kComputeWarps; ++w) {
                            const int cu = w % kColBlocks, j = w / kColBlocks;
                            const bool want = act && cv0 <= cv1 && cu >= cu0 && cu <= cu1 &&
                                              j >= j0 && j <= j1;
                            const uint32_t bal = __ballot_sync(0xffffffffu, want);
                            if (!bal) continue;
                            int pos0 = 0;
                            const int leader = __ffs(bal) - 1;
                            if (lane == leader) pos0 = atomicAdd(&sm.cnt[buf][w], __popc(bal));
                            pos0 = __shfl_sync(0xffffffffu, pos0, leader);
                            if (want) sm.list[buf][w][pos0 + __popc(bal & ((1u << lane) - 1u))] = make_int2(base, (int)vidc);
                        }
                    }
                    if (pw == 0 && lane == 0) {
                        sm.tile[buf] = item.tile;
                        sm.last[buf] = (b == nb_total - 1);
                    }
                }
                __syncwarp();
                __threadfence_block();
                bar_arrive(1 + buf, kSyncThreads);  // this warp's part of the batch is ready
                buf = (buf + 1) % kBufs;
                ++uses;
            }
            if (done) {
                // complete the consumers' last releases of the other buffers so
                // that every barrier generation is balanced before exit
                // (batch k was released by the consumers for k < E = uses - 1;
                // the producer already waited on releases of k <= E - kBufs)
                for (int k = max(0, uses - kBufs); k <= uses - 2; ++k)
                    bar_sync(1 + kBufs + (k % kBufs), kSyncThreads);
                break;
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int bu = (warp % kColBlocks) * 8, bv = (warp / kColBlocks) * 4;
    const int lu = lane & 7, lv = lane >> 3;
    const float2* __restrict__ tab = a.ptable + (bv + lv) * SP + bu + lu;
    const int N = a.N;
    // Separate accumulators for records with the kernel (n) and with its
    // conjugate (c, w < 0), with P = sum K (.) V and Q = sum (K.y, K.x) (.) V:
    //   K V       : re = P.x - P.y,  im = Q.x + Q.y
    //   conj(K) V : re = P.x + P.y,  im = Q.y - Q.x
    float2 Pn[NPOL], Qn[NPOL], Pc[NPOL], Qc[NPOL];
#pragma unroll
    for (int p = 0; p < NPOL; ++p) Pn[p] = Qn[p] = Pc[p] = Qc[p] = make_float2(0.f, 0.f);

    struct Stage {
        float2 K;
        float2 V[NPOL];
        uint32_t conj;
    };
    auto load_stage = [&](Stage& st, int2 e) {
        st.K = __ldg(tab + e.x);
        const uint32_t vid = (uint32_t)e.y & 0x7fffffffu;
        st.conj = (uint32_t)e.y >> 31;
        const float2* vp = a.vis + (size_t)vid * NPOL;
        if constexpr (NPOL % 2 == 0) {
#pragma unroll
            for (int p = 0; p < NPOL; p += 2) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(vp + p));
                st.V[p] = make_float2(q.x, q.y);
                st.V[p + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int p = 0; p < NPOL; ++p) st.V[p] = __ldg(vp + p);
        }
    };
    auto fma_stage = [&](const Stage& st) {
        const float2 Ks = make_float2(st.K.y, st.K.x);
        if (st.conj) {
#pragma unroll
            for (int p = 0; p < NPOL; ++p) {
                Pc[p] = __ffma2_rn(st.K, st.V[p], Pc[p]);
                Qc[p] = __ffma2_rn(Ks, st.V[p], Qc[p]);
            }
        } else {
#pragma unroll
            for (int p = 0; p < NPOL; ++p) {
                Pn[p] = __ffma2_rn(st.K, st.V[p], Pn[p]);
                Qn[p] = __ffma2_rn(Ks, st.V[p], Qn[p]);
            }
        }
    };

    int buf = 0;
    for (;;) {
        bar_sync(1 + buf, kSyncThreads);  // wait for the batch
        const int tile = sm.tile[buf];
        if (tile < 0) break;
        const int last = sm.last[buf];
        const int n = sm.cnt[buf][warp];
        const int2* lst = sm.list[buf][warp];
        // three-stage pipeline: kernel values and visibilities of the next two
        // entries are in flight while one entry's multiply-adds issue
        Stage A, B, C;
        if (n > 0) load_stage(A, lst[0]);
        if (n > 1) load_stage(B, lst[1]);
        int i = 0;
        for (; i + 2 < n; i += 3) {
            load_stage(C, lst[i + 2]);
            fma_stage(A);
            if (i + 3 < n) load_stage(A, lst[i + 3]);
            fma_stage(B);
            if (i + 4 < n) load_stage(B, lst[i + 4]);
            fma_stage(C);
        }
        if (i < n) fma_stage(A);
        if (i + 1 < n) fma_stage(B);
        if (last) {
            // commit the block's accumulators of this work item
            const int u = (tile % side_u) * kTileU + bu + lu;
            const int v = (tile / side_u) * kTileV + bv + lv;
#pragma unroll
            for (int p = 0; p < NPOL; ++p) {
                const float re = (Pn[p].x - Pn[p].y) + (Pc[p].x + Pc[p].y);
                const float im = (Qn[p].x + Qn[p].y) + (Qc[p].y - Qc[p].x);
                if (u < N && v < N && (re != 0.f || im != 0.f))
                    atomicAdd(a.grid + ((int64_t)p * N + v) * N + u, make_float2(re, im));
                Pn[p] = Qn[p] = Pc[p] = Qc[p] = make_float2(0.f, 0.f);
            }
        }
        bar_arrive(1 + kBufs + buf, kSyncThreads);  // buffer free
        buf = (buf + 1) % kBufs;
    }
}

template <int NPOL, int SP>
void launch_sp(const GridArgs& a, int num_sms, cudaStream_t s) {
    const size_t smem = sizeof(Smem<NPOL>);
    cudaFuncSetAttribute(k_grid<NPOL, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid<NPOL, SP>, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    k_grid<NPOL, SP><<<num_sms * per_sm, kThreads, smem, s>>>(a);
    note_launch();
}

template <int NPOL>
void launch_t(const GridArgs& a, int num_sms, cudaStream_t s) {
    switch (a.pad_stride) {
        case 24: launch_sp<NPOL, 24>(a, num_sms, s); break;
        case 32: launch_sp<NPOL, 32>(a, num_sms, s); break;
        case 48: launch_sp<NPOL, 48>(a, num_sms, s); break;
        case 80: launch_sp<NPOL, 80>(a, num_sms, s); break;
        case 144: launch_sp<NPOL, 144>(a, num_sms, s); break;
        default: launch_sp<NPOL, 272>(a, num_sms, s); break;
    }
}

// Zero-padded copy of the tables: slice (p, o) becomes (S + 6) rows x SP
// columns with the S x S values at row 3, column 7.
__global__ void k_pad_tables(const float2* __restrict__ tab, const int64_t* __restrict__ plane_off,
                             const int64_t* __restrict__ pplane_off, const int* __restrict__ support,
                             int P, int beta, int SP, float2* __restrict__ ptab) {
    const int p = blockIdx.y;
    if (p >= P) return;
    const int S = support[p], SR = S + 6;
    const int64_t per = (int64_t)SR * SP;
    const int64_t n = (int64_t)beta * beta * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = e / per;
        const int rem = (int)(e - o * per);
        const int row = rem / SP - 3, col = rem % SP - 7;
        float2 v = make_float2(0.f, 0.f);
        if (row >= 0 && row < S && col >= 0 && col < S)
            v = tab[plane_off[p] + o * S * S + (int64_t)row * S + col];
        ptab[pplane_off[p] + e] = v;
    }
}

__global__ void k_weight_vis(const float2* __restrict__ vis, const float* __restrict__ w,
                             int64_t n, float2* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = vis[e];
        const float s = w[e];
        out[e] = make_float2(v.x * s, v.y * s);
    }
}

}  // namespace

void launch_weight_vis(const float2* vis, const float* w, int64_t n, float2* out, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_weight_vis<<<(unsigned)blocks, 256, 0, s>>>(vis, w, n, out);
    note_launch();
}

int padded_stride(int smax) {
    const int need = smax + 14;
    for (int sp : {24, 32, 48, 80, 144}) if (need <= sp) return sp;
    return 272;
}

int64_t padded_table_elems(int S, int beta, int SP) { return (int64_t)beta * beta * (S + 6) * SP; }

void launch_pad_tables(const float2* tab, const int64_t* plane_off, const int64_t* pplane_off,
                       const int* support, int P, int beta, int SP, float2* ptab, cudaStream_t s) {
    k_pad_tables<<<dim3(256, P), 256, 0, s>>>(tab, plane_off, pplane_off, support, P, beta, SP, ptab);
    note_launch();
}

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
