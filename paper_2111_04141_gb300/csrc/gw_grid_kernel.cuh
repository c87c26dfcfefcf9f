// Gridding kernel: w-projection convolutional gridding onto a complex grid.
// Included once per table kind by gw_grid_c64.cu, gw_grid_bf16.cu and
// gw_grid_f16.cu.
//
// Computes the Gridding Step of Algorithm convgriddingoversampling
// (Section 2.4.5) with the w-projection GCF (Section 1.7.1):
//     G[pol][kv + tv][ku + tu] += K_p[ov][ou](tv, tu) * V[pol]   (conj K if w < 0)
//
// Design (GB300):
// * A CTA owns one 32 x 32 tile of the grid for a work item (a run of that
//   tile's bin) and keeps the tile's accumulators in registers, so each grid
//   point is committed once per work item (vector atomics, red.global).
//   Two CTAs run per SM.
// * Eight compute warps each own an 8 (u) x 16 (v) block; lane (lu, lv) holds
//   the points (lu, lv + 4 j), j = 0..3 ("slots" of 8 x 4 points), for every
//   polarisation.  Four slots per warp amortise each record's staged
//   visibility over up to 4 x 32 points.
// * A ninth, producer warp stages batches of records into shared memory
//   (three buffers, handed over with named barriers) and, for every record,
//   appends it to the list of each compute warp whose block its footprint
//   meets, together with the record's table offset for the tile and the
//   range of slots its rows meet (one 64-bit entry).  Compute warps
//   therefore only see records that touch them.
// * Kernel values come from zero-padded slices (7 zero columns and 3 zero
//   rows around each S x S slice, one compile-time row stride per plan), so
//   lanes outside the footprint read zeros and slot addresses are immediate
//   offsets; loads for the next record are issued before the multiply-adds
//   of the current one.
// * Per tap and polarisation the update is two packed FP32x2 FMAs (Blackwell
//   FFMA2) on the (re, im) accumulator pair:
//     acc += (K.re, K.re) (.) A + (K.im, K.im) (.) B
//   with A = V and B = (-V.im, V.re), or (V.im, -V.re) for the conjugate
//   kernel (w < 0), precomputed per record.
// * Storage precision: the table element type is a template parameter
//   (complex FP32, or bfloat16 / float16 pairs widened to FP32 on load);
//   visibilities of any kind are widened to FP32 when staged; all
//   accumulation is FP32.  With an error grid the commit is compensated
//   (commit_compensated).
#pragma once

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kComputeWarps = 8;
constexpr int kThreads = (kComputeWarps + 1) * 32;
constexpr int kBatch = 256;

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

// Commit with the rounding error kept: the vector atomic returns the value
// it added to, so the exact error of the (round-to-nearest) sum it stored is
// recovered with Knuth's TwoSum and accumulated into a second grid.  The
// compensated value is grid + err (a Kahan-style sum of the commits).
__device__ __forceinline__ void commit_compensated(float2* g, float2* err, float2 val) {
    const float2 old = atomicAdd(g, val);
    float2 e;
    {
        const float s = __fadd_rn(old.x, val.x);
        const float bv = __fsub_rn(s, old.x);
        const float av = __fsub_rn(s, bv);
        e.x = __fadd_rn(__fsub_rn(old.x, av), __fsub_rn(val.x, bv));
    }
    {
        const float s = __fadd_rn(old.y, val.y);
        const float bv = __fsub_rn(s, old.y);
        const float av = __fsub_rn(s, bv);
        e.y = __fadd_rn(__fsub_rn(old.y, av), __fsub_rn(val.y, bv));
    }
    if (e.x != 0.f || e.y != 0.f) atomicAdd(err, e);
}

template <int NPOL, int B>
struct Smem {
    float4 v[B][kBatch][NPOL];             // (A.re, A.im, B.re, B.im) per polarisation
    // per warp: entries (x: padded-table index of the tile origin relative to
    // the record, y: r | j0 << 16 | j1 << 20), those meeting all four slots
    // from the front, the others from the back
    uint2 list[B][kComputeWarps][kBatch];
    int cnt[B][kComputeWarps];             // entries meeting all four slots
    int cntp[B][kComputeWarps];            // entries meeting some slots
    int tile[B];                           // tile of the batch; -1 = end of work
    int last[B];                           // batch ends its work item
};

// Packed FMAs of one entry into slots J0..J1 (compile-time range).
template <int NPOL, int J0, int J1>
__device__ __forceinline__ void slot_fma(float2 (&acc)[4][NPOL], const float2 (&Kc)[4],
                                         const float4 (&V)[NPOL]) {
#pragma unroll
    for (int j = J0; j <= J1; ++j) {
        const float2 kxx = make_float2(Kc[j].x, Kc[j].x);
        const float2 kyy = make_float2(Kc[j].y, Kc[j].y);
#pragma unroll
        for (int p = 0; p < NPOL; ++p) {
            acc[j][p] = __ffma2_rn(kxx, make_float2(V[p].x, V[p].y), acc[j][p]);
            acc[j][p] = __ffma2_rn(kyy, make_float2(V[p].z, V[p].w), acc[j][p]);
        }
    }
}

// One warp's pass over n list entries of a batch.  Software pipeline: the
// kernel values of entry i + 1 load while entry i's FMAs run (a ring of D
// register sets, unrolled so no register copies are needed).  FULL: every
// entry meets all four slots of the warp's block (no per-slot tests);
// otherwise one warp-uniform jump on the entry's slot range selects code
// for exactly the slots it meets.
template <int NPOL, int SP, int D, bool FULL, class TE>
__device__ __forceinline__ void run_entries(const uint2* lst, int n,
                                            const float4 (*vs)[NPOL],
                                            const typename TE::T* __restrict__ tab,
                                            float2 (&acc)[4][NPOL]) {
    float2 Kr[D][4];
    uint32_t er[D];
    auto load_k = [&](uint2 en, float2 (&K)[4]) {
        const uint32_t e = en.y;
        const typename TE::T* p_ = tab + (int)en.x;
        if (FULL) {
            K[0] = TE::load(p_);
            K[1] = TE::load(p_ + 4 * SP);
            K[2] = TE::load(p_ + 8 * SP);
            K[3] = TE::load(p_ + 12 * SP);
        } else {
            const int j0_ = (e >> 16) & 15, j1_ = (e >> 20) & 15;
            K[0] = K[1] = K[2] = K[3] = make_float2(0.f, 0.f);
            if (0 >= j0_ && 0 <= j1_) K[0] = TE::load(p_);
            if (1 >= j0_ && 1 <= j1_) K[1] = TE::load(p_ + 4 * SP);
            if (2 >= j0_ && 2 <= j1_) K[2] = TE::load(p_ + 8 * SP);
            if (3 >= j0_ && 3 <= j1_) K[3] = TE::load(p_ + 12 * SP);
        }
    };
#pragma unroll
    for (int d = 0; d < D; ++d) {
        er[d] = 0;
        Kr[d][0] = Kr[d][1] = Kr[d][2] = Kr[d][3] = make_float2(0.f, 0.f);
        if (d < n) {
            const uint2 en = lst[d];
            er[d] = en.y;
            load_k(en, Kr[d]);
        }
    }
    for (int i = 0; i < n; i += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (i + d < n) {
                const uint32_t ec = er[d];
                const float2 Kc[4] = {Kr[d][0], Kr[d][1], Kr[d][2], Kr[d][3]};
                if (i + d + D < n) {
                    const uint2 en = lst[i + d + D];
                    er[d] = en.y;
                    load_k(en, Kr[d]);
                }
                const int r = ec & 0xffff, j0 = (ec >> 16) & 15, j1 = (ec >> 20) & 15;
                float4 V[NPOL];
#pragma unroll
                for (int p = 0; p < NPOL; ++p) V[p] = vs[r][p];
                // packed FP32x2: acc += (K.x, K.x) (.) A + (K.y, K.y) (.) B, only
                // on the slots the entry meets (one warp-uniform jump)
                if (FULL) {
                    slot_fma<NPOL, 0, 3>(acc, Kc, V);
                } else {
                    switch ((j0 << 2) | j1) {
                        case 0: slot_fma<NPOL, 0, 0>(acc, Kc, V); break;
                        case 1: slot_fma<NPOL, 0, 1>(acc, Kc, V); break;
                        case 2: slot_fma<NPOL, 0, 2>(acc, Kc, V); break;
                        case 3: slot_fma<NPOL, 0, 3>(acc, Kc, V); break;
                        case 5: slot_fma<NPOL, 1, 1>(acc, Kc, V); break;
                        case 6: slot_fma<NPOL, 1, 2>(acc, Kc, V); break;
                        case 7: slot_fma<NPOL, 1, 3>(acc, Kc, V); break;
                        case 10: slot_fma<NPOL, 2, 2>(acc, Kc, V); break;
                        case 11: slot_fma<NPOL, 2, 3>(acc, Kc, V); break;
                        default: slot_fma<NPOL, 3, 3>(acc, Kc, V); break;
                    }
                }
            }
        }
    }
}

// Named barriers: FULL(b) = 1 + b (batch b staged), EMPTY(b) = 1 + B + b (consumed).
template <int NPOL, int SP, int TK, int D, int B>
__global__ void __launch_bounds__(kThreads, 2) k_grid(GridArgs a) {
    using TE = TabElem<TK>;
    constexpr int kBufs = B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<NPOL, B>& sm = *reinterpret_cast<Smem<NPOL, B>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int side = a.ntiles_u;
    const int hb = a.beta / 2;

    if (warp == kComputeWarps) {
        // ------------------------------------------------------------ producer
        const uint32_t nitems = *a.item_count;
        int buf = 0, uses = 0;
        for (;;) {
            uint32_t it = 0;
            if (lane == 0) it = atomicAdd(a.queue, 1u);
            it = __shfl_sync(0xffffffffu, it, 0);
            const bool done = it >= nitems;
            Item item{};
            if (!done) item = a.items[it];
            const int nb_total = done ? 1 : (item.len + kBatch - 1) / kBatch;
            for (int b = 0; b < nb_total; ++b) {
                if (uses >= kBufs) bar_sync(1 + kBufs + buf, kThreads);  // wait until consumed
                if (lane < kComputeWarps) {
                    sm.cnt[buf][lane] = 0;
                    sm.cntp[buf][lane] = 0;
                }
                __syncwarp();
                if (done) {
                    if (lane == 0) {
                        sm.tile[buf] = -1;
                        sm.last[buf] = 1;
                    }
                } else {
                    // with w-layers (w-stacking) a tile id is layer * layer_tiles + tile
                    const int ltile = a.layer_tiles ? item.tile % a.layer_tiles : item.tile;
                    const int tu0 = (ltile % side) * kTile;
                    const int tv0 = (ltile / side) * kTile;
                    const int b0 = b * kBatch;
                    const int nb = min(kBatch, item.len - b0);
                    for (int r = lane; r < nb; r += 32) {
                        const uint32_t id = __ldg(a.entries + item.start + b0 + r);
                        const gw_index_rec rc = load_rec(a.rec, id);
                        // w-stacking records carry their layer in `plane`; the
                        // kernel is the plan's single (w = 0) plane
                        const int plane = a.layer_tiles ? 0 : rc.plane;
                        const int S = __ldg(a.support + plane), h = S >> 1;
                        const int64_t slice = __ldg(a.pplane_off + plane) +
                                              ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) *
                                                  (int64_t)(S + 6) * SP;
                        // padded index of the tile origin relative to this record
                        const int base = (int)slice + (tv0 - rc.kv + h + 3) * SP + (tu0 - rc.ku + h + 7);
                        const bool conj = (rc.flags & GW_FLAG_CONJ) != 0;
#pragma unroll
                        for (int p = 0; p < NPOL; ++p) {
                            float2 v = load_vis(a.vis, a.vis_kind, (int64_t)id * NPOL + p);
                            if (a.weight) {
                                const float w = __ldg(a.weight + (int64_t)id * NPOL + p);
                                v.x *= w;
                                v.y *= w;
                            }
                            sm.v[buf][r][p] = conj ? make_float4(v.x, v.y, v.y, -v.x)
                                                   : make_float4(v.x, v.y, -v.y, v.x);
                        }
                        // footprint relative to the tile: [ulo, uhi] x [vlo, vhi]
                        const int ulo = rc.ku - h - tu0, uhi = rc.ku + h - tu0;
                        const int vlo = rc.kv - h - tv0, vhi = rc.kv + h - tv0;
                        const int cu0 = max(0, ulo) >> 3, cu1 = min(kTile - 1, uhi) >> 3;
                        const int cv0 = max(0, vlo) >> 4, cv1 = min(kTile - 1, vhi) >> 4;
                        for (int cv = cv0; cv <= cv1; ++cv) {
                            const int j0 = max(0, vlo - 16 * cv) >> 2;
                            const int j1 = min(15, vhi - 16 * cv) >> 2;
                            const uint2 e = make_uint2((uint32_t)base,
                                                       (uint32_t)r | ((uint32_t)j0 << 16) | ((uint32_t)j1 << 20));
                            const bool full = j0 == 0 && j1 == 3;
                            for (int cu = cu0; cu <= cu1; ++cu) {
                                const int w = cv * 4 + cu;
                                if (full) {
                                    const int pos = atomicAdd(&sm.cnt[buf][w], 1);
                                    sm.list[buf][w][pos] = e;
                                } else {
                                    const int pos = atomicAdd(&sm.cntp[buf][w], 1);
                                    sm.list[buf][w][kBatch - 1 - pos] = e;
                                }
                            }
                        }
                    }
                    if (lane == 0) {
                        sm.tile[buf] = item.tile;
                        sm.last[buf] = (b == nb_total - 1);
                    }
                }
                __syncwarp();
                __threadfence_block();
                bar_arrive(1 + buf, kThreads);  // batch ready
                buf = (buf + 1 == kBufs) ? 0 : buf + 1;
                ++uses;
            }
            if (done) {
                // complete the consumers' releases of the batches whose
                // buffers were not reused, so every barrier generation is
                // balanced before exit (the end-of-work batch is not released)
                for (int q = max(0, uses - kBufs); q <= uses - 2; ++q)
                    bar_sync(1 + kBufs + q % kBufs, kThreads);
                break;
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int bu = (warp & 3) * 8, bv = (warp >> 2) * 16;
    const int lu = lane & 7, lv = lane >> 3;
    const typename TE::T* __restrict__ tab =
        reinterpret_cast<const typename TE::T*>(a.ptable) + (bv + lv) * SP + bu + lu;
    const int N = a.N;
    float2 acc[4][NPOL];   // (re, im)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int p = 0; p < NPOL; ++p) acc[j][p] = make_float2(0.f, 0.f);

    int buf = 0;
    for (;;) {
        bar_sync(1 + buf, kThreads);  // wait for the batch
        const int tile = sm.tile[buf];
        if (tile < 0) break;
        const int last = sm.last[buf];
        const int nf = sm.cnt[buf][warp], np = sm.cntp[buf][warp];
        const uint2* lst = sm.list[buf][warp];
        // entries meeting all four slots: no per-slot tests
        run_entries<NPOL, SP, D, true, TE>(lst, nf, sm.v[buf], tab, acc);
        // entries meeting a subset of the slots
        run_entries<NPOL, SP, D, false, TE>(lst + kBatch - np, np, sm.v[buf], tab, acc);
        if (last) {
            // commit the tile's accumulators of this work item
            const int ltile = a.layer_tiles ? tile % a.layer_tiles : tile;
            float2* const gbase = a.grid + (a.layer_tiles ? (int64_t)(tile / a.layer_tiles) *
                                                                 a.layer_stride : 0);
            const int u = (ltile % a.ntiles_u) * kTile + bu + lu;
            const int v0 = (ltile / a.ntiles_u) * kTile + bv + lv;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int v = v0 + 4 * j;
#pragma unroll
                for (int p = 0; p < NPOL; ++p) {
                    if (u < N && v < N && (acc[j][p].x != 0.f || acc[j][p].y != 0.f)) {
                        const float2 val = make_float2(acc[j][p].x * a.table_inv,
                                                       acc[j][p].y * a.table_inv);
                        const int64_t off = ((int64_t)p * N + v) * N + u;
                        if (a.grid_err) {
                            commit_compensated(gbase + off, a.grid_err + off, val);
                        } else {
                            atomicAdd(gbase + off, val);
                        }
                    }
                    acc[j][p] = make_float2(0.f, 0.f);
                }
            }
        }
        bar_arrive(1 + kBufs + buf, kThreads);  // buffer free
        buf = (buf + 1 == kBufs) ? 0 : buf + 1;
    }
}

template <int NPOL, int SP, int TK, int D, int B>
void launch_v(const GridArgs& a, int num_sms, cudaStream_t s) {
    const size_t smem = sizeof(Smem<NPOL, B>);
    cudaFuncSetAttribute(k_grid<NPOL, SP, TK, D, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid<NPOL, SP, TK, D, B>, kThreads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    k_grid<NPOL, SP, TK, D, B><<<num_sms * per_sm, kThreads, smem, s>>>(a);
    note_launch();
}

// Two register sets of kernel values in flight and three staging buffers of
// 256 records: measured fastest on the 4-pol w-projection workload among
// rings of 2-4 entries, 2-4 buffers and batches of 128-256 records (deeper
// rings raise register pressure; a fourth buffer does not fit two CTAs per
// SM with 64-bit list entries).
template <int NPOL, int SP, int TK>
void launch_sp(const GridArgs& a, int num_sms, cudaStream_t s) {
    launch_v<NPOL, SP, TK, 2, 3>(a, num_sms, s);
}

template <int NPOL, int TK>
void launch_t(const GridArgs& a, int num_sms, cudaStream_t s) {
    switch (a.pad_stride) {
        case 24: launch_sp<NPOL, 24, TK>(a, num_sms, s); break;
        case 32: launch_sp<NPOL, 32, TK>(a, num_sms, s); break;
        case 48: launch_sp<NPOL, 48, TK>(a, num_sms, s); break;
        case 80: launch_sp<NPOL, 80, TK>(a, num_sms, s); break;
        case 144: launch_sp<NPOL, 144, TK>(a, num_sms, s); break;
        default: launch_sp<NPOL, 272, TK>(a, num_sms, s); break;
    }
}

}  // namespace

// All gridder instantiations for one table kind.
template <int TK>
void launch_grid_kind(const GridArgs& a, int num_sms, cudaStream_t s) {
    switch (a.npol) {
        case 1: launch_t<1, TK>(a, num_sms, s); break;
        case 2: launch_t<2, TK>(a, num_sms, s); break;
        case 3: launch_t<3, TK>(a, num_sms, s); break;
        default: launch_t<4, TK>(a, num_sms, s); break;
    }
}


}  // namespace gw
