// Gridding kernel: w-projection convolutional gridding onto a complex grid.
//
// Computes the Gridding Step of Algorithm convgriddingoversampling
// (Section 2.4.5) with the w-projection GCF (Section 1.7.1):
//     G[pol][kv + tv][ku + tu] += K_p[ov][ou](tv, tu) * V[pol]   (conj K if w < 0)
//
// Design (GB300):
// * A CTA owns one kTile x kTile tile of the grid for a work item (a run of
//   that tile's bin) and keeps the tile's accumulators in registers, so each
//   grid point is committed once per work item (vector atomics, red.global).
// * The tile is 64 (u) x 32 (v).  Eight compute warps each own an 8 (u) x
//   32 (v) column; lane (lu, lv) holds the points (lu, lv + 4 j), j = 0..7
//   ("slots" of 8 x 4 points), for every polarisation.
// * A fifth warpgroup of four producer warps (handing registers to the
//   consumers with setmaxnreg) stages batches of records into shared memory
//   (four batches in flight, handed over with named barriers) and, for every record,
//   appends it to the list of each compute warp whose block its footprint
//   meets, together with the range of slots its rows meet.  Compute warps
//   therefore only see records that touch them, and skip untouched slots with
//   one uniform test.
// * Kernel values come from zero-padded slices (7 zero columns and 3 zero
//   rows around each S x S slice, one compile-time row stride per plan), so
//   lanes outside the footprint read zeros without predication and slot
//   addresses are immediate offsets; loads for the next record are issued
//   before the multiply-adds of the current one (ping-pong registers).
// * Per tap and polarisation the complex update costs two packed FP32x2 FMAs
//   (Blackwell FFMA2: two multiply-adds per issued instruction, so control
//   instructions issue in the FMA pipe's spare slots).  Without broadcasting K:
//     P += K (.) (V.x, -s V.y),  Q += K (.) (V.y, s V.x),
//     re = P.x + P.y,  im = Q.x + Q.y   at commit,
//   s = +1, or -1 for records with w < 0 (conj(K) V), folded into the staged
//   visibility so mixed records share accumulators.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kComputeWarps = 8;
// Two consumer warpgroups plus one producer warpgroup of four warps.
// Register split (setmaxnreg): launched at 168 per thread; the producers give
// back to 40, the consumers take 232:
// 128 x 40 + 256 x 232 = 64512 = 384 x 168.
constexpr int kThreads = (kComputeWarps + 4) * 32;
constexpr int kSyncThreads = kThreads;                   // threads in the batch barriers
constexpr int kProducerThreads = 4 * 32;                 // producer-only barrier (id 9)
constexpr int kProducerRegs = 40, kConsumerRegs = 232;
constexpr int kBatch = 256;
constexpr int kBufs = 4;             // batches in flight (barriers 1..4 full, 5..8 empty)
constexpr int kSlots = 8;            // 8 x 4-row slots: a warp block is 8 (u) x 32 (v)
constexpr int kTileU = 64, kTileV = 32;
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
    int rec[kBufs][kBatch];                // padded-table index of the tile origin for the record
    float4 v[kBufs][kBatch][NPOL];         // (V.x, -s V.y, V.y, s V.x), s = -1 for w < 0
    uint32_t list[kBufs][kComputeWarps][kBatch];  // record | first slot << 8 | last slot << 11
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
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
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
                        uint32_t e = 0;
                        int cu0 = 1, cu1 = 0, cv0 = 1, cv1 = 0, vlo = 0, vhi = -1;
                        if (act) {
                            const uint32_t id = __ldg(a.entries + item.start + b0 + r);
                            const gw_index_rec rc = load_rec(a.rec, id);
                            const int S = __ldg(a.support + rc.plane), h = S >> 1;
                            const int64_t slice = __ldg(a.pplane_off + rc.plane) +
                                                  ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) *
                                                      (int64_t)(S + 6) * SP;
                            // padded index of the tile origin relative to this record
                            sm.rec[buf][r] = (int)slice + (tv0 - rc.kv + h + 3) * SP + (tu0 - rc.ku + h + 7);
                            const float sg = (rc.flags & GW_FLAG_CONJ) ? -1.f : 1.f;
                            float2 v[NPOL];
#pragma unroll
                            for (int p = 0; p < NPOL; ++p) v[p] = __ldg(a.vis + (int64_t)id * NPOL + p);
                            if (a.weight) {
#pragma unroll
                                for (int p = 0; p < NPOL; ++p) {
                                    const float w = __ldg(a.weight + (int64_t)id * NPOL + p);
                                    v[p].x *= w;
                                    v[p].y *= w;
                                }
                            }
#pragma unroll
                            for (int p = 0; p < NPOL; ++p)
                                sm.v[buf][r][p] = make_float4(v[p].x, -sg * v[p].y, v[p].y, sg * v[p].x);
                            // footprint relative to the tile
                            const int ulo = rc.ku - h - tu0, uhi = rc.ku + h - tu0;
                            vlo = rc.kv - h - tv0;
                            vhi = rc.kv + h - tv0;
                            cu0 = max(0, ulo) >> 3;
                            cu1 = min(kTileU - 1, uhi) >> 3;
                            cv0 = 0;
                            cv1 = (vhi >= 0 && vlo <= kTileV - 1) ? 0 : -1;
                            e = (uint32_t)r;
                        }
                        // warp-aggregated appends: one shared atomic per target warp
                        {
                            const bool in_v = act && cv0 <= cv1;
                            const int j0 = max(0, vlo) >> 2;
                            const int j1 = min(kTileV - 1, vhi) >> 2;
                            const uint32_t jr = in_v ? ((uint32_t)j0 | ((uint32_t)j1 << 3)) : 0u;
                            for (int cu = 0; cu < kTileU / 8; ++cu) {
                                const bool want = in_v && cu >= cu0 && cu <= cu1;
                                const uint32_t bal = __ballot_sync(0xffffffffu, want);
                                if (!bal) continue;
                                const int w = cu;
                                int base = 0;
                                const int leader = __ffs(bal) - 1;
                                if (lane == leader) base = atomicAdd(&sm.cnt[buf][w], __popc(bal));
                                base = __shfl_sync(0xffffffffu, base, leader);
                                if (want)
                                    sm.list[buf][w][base + __popc(bal & ((1u << lane) - 1u))] = e | (jr << 8);
                            }
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
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegs));
    const int bu = warp * 8;
    const int lu = lane & 7, lv = lane >> 3;
    const float2* __restrict__ tab = a.ptable + lv * SP + bu + lu;
    const int N = a.N;
    // P = sum K (.) (V.x, -s V.y), Q = sum K (.) (V.y, s V.x):
    // re = P.x + P.y, im = Q.x + Q.y  (s = -1 for the conjugate kernel)
    float2 P[kSlots][NPOL], Q[kSlots][NPOL];
#pragma unroll
    for (int j = 0; j < kSlots; ++j)
#pragma unroll
        for (int p = 0; p < NPOL; ++p) P[j][p] = Q[j][p] = make_float2(0.f, 0.f);

    // Active slots of an entry are the contiguous range [j0, j1]: a switch on
    // j0 falls through the slots and breaks after j1, so inactive slots issue
    // nothing (no predicated-off work).
#define GW_LOAD_SLOT(K, p_, j) K[j] = __ldg((p_) + (j) * 4 * SP)
#define GW_LOAD(K, e)                                                          \
    do {                                                                       \
        const float2* p_ = tab + sm.rec[buf][(e) & 0xff];                      \
        const int j0_ = ((e) >> 8) & 7, j1_ = ((e) >> 11) & 7;                 \
        switch (j0_) {                                                         \
            case 0: GW_LOAD_SLOT(K, p_, 0); if (j1_ == 0) break;               \
            case 1: GW_LOAD_SLOT(K, p_, 1); if (j1_ == 1) break;               \
            case 2: GW_LOAD_SLOT(K, p_, 2); if (j1_ == 2) break;               \
            case 3: GW_LOAD_SLOT(K, p_, 3); if (j1_ == 3) break;               \
            case 4: GW_LOAD_SLOT(K, p_, 4); if (j1_ == 4) break;               \
            case 5: GW_LOAD_SLOT(K, p_, 5); if (j1_ == 5) break;               \
            case 6: GW_LOAD_SLOT(K, p_, 6); if (j1_ == 6) break;               \
            default: GW_LOAD_SLOT(K, p_, 7);                                    \
        }                                                                      \
    } while (0)
#define GW_FMA_SLOT(K, j)                                                      \
    _Pragma("unroll") for (int p = 0; p < NPOL; ++p) {                         \
        P[j][p] = __ffma2_rn(K[j], make_float2(V[p].x, V[p].y), P[j][p]);      \
        Q[j][p] = __ffma2_rn(K[j], make_float2(V[p].z, V[p].w), Q[j][p]);      \
    }
#define GW_FMA(K, e)                                                           \
    do {                                                                       \
        const float4* v_ = sm.v[buf][(e) & 0xff];                              \
        float4 V[NPOL];                                                        \
        _Pragma("unroll") for (int p = 0; p < NPOL; ++p) V[p] = v_[p];         \
        const int j0_ = ((e) >> 8) & 7, j1_ = ((e) >> 11) & 7;                 \
        switch (j0_) {                                                         \
            case 0: GW_FMA_SLOT(K, 0) if (j1_ == 0) break;                     \
            case 1: GW_FMA_SLOT(K, 1) if (j1_ == 1) break;                     \
            case 2: GW_FMA_SLOT(K, 2) if (j1_ == 2) break;                     \
            case 3: GW_FMA_SLOT(K, 3) if (j1_ == 3) break;                     \
            case 4: GW_FMA_SLOT(K, 4) if (j1_ == 4) break;                     \
            case 5: GW_FMA_SLOT(K, 5) if (j1_ == 5) break;                     \
            case 6: GW_FMA_SLOT(K, 6) if (j1_ == 6) break;                     \
            default: GW_FMA_SLOT(K, 7)                                          \
        }                                                                      \
    } while (0)

    int buf = 0;
    for (;;) {
        bar_sync(1 + buf, kSyncThreads);  // wait for the batch
        const int tile = sm.tile[buf];
        if (tile < 0) break;
        const int last = sm.last[buf];
        const int n = sm.cnt[buf][warp];
        const uint32_t* lst = sm.list[buf][warp];
        // three-stage pipeline over the warp's entries: kernel values of the
        // next two entries are in flight while one entry's multiply-adds issue
        float2 KA[kSlots], KB[kSlots], KC[kSlots];
        uint32_t eA = 0, eB = 0, eC = 0;
        if (n > 0) { eA = lst[0]; GW_LOAD(KA, eA); }
        if (n > 1) { eB = lst[1]; GW_LOAD(KB, eB); }
        int i = 0;
        for (; i + 2 < n; i += 3) {
            eC = lst[i + 2];
            GW_LOAD(KC, eC);
            GW_FMA(KA, eA);
            if (i + 3 < n) { eA = lst[i + 3]; GW_LOAD(KA, eA); }
            GW_FMA(KB, eB);
            if (i + 4 < n) { eB = lst[i + 4]; GW_LOAD(KB, eB); }
            GW_FMA(KC, eC);
        }
        if (i < n) GW_FMA(KA, eA);
        if (i + 1 < n) GW_FMA(KB, eB);
        if (last) {
            // commit the tile's accumulators of this work item
            const int u = (tile % side_u) * kTileU + bu + lu;
            const int v0 = (tile / side_u) * kTileV + lv;
#pragma unroll
            for (int j = 0; j < kSlots; ++j) {
                const int v = v0 + 4 * j;
#pragma unroll
                for (int p = 0; p < NPOL; ++p) {
                    const float re = P[j][p].x + P[j][p].y, im = Q[j][p].x + Q[j][p].y;
                    if (u < N && v < N && (re != 0.f || im != 0.f))
                        atomicAdd(a.grid + ((int64_t)p * N + v) * N + u, make_float2(re, im));
                    P[j][p] = Q[j][p] = make_float2(0.f, 0.f);
                }
            }
        }
        bar_arrive(1 + kBufs + buf, kSyncThreads);  // buffer free
        buf = (buf + 1) % kBufs;
    }
#undef GW_LOAD
#undef GW_LOAD_SLOT
#undef GW_FMA
#undef GW_FMA_SLOT
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

}  // namespace

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
