// Gridding kernel: w-projection convolutional gridding onto a complex grid.
// Included once per table kind by gw_grid_c64.cu, gw_grid_bf16.cu and
// gw_grid_f16.cu.
//
// Computes the Gridding Step of Algorithm convgriddingoversampling
// (Section 2.4.5) with the w-projection GCF (Section 1.7.1):
//     G[pol][kv + tv][ku + tu] += K_p[ov][ou](tv, tu) * V[pol]   (conj K if w < 0)
//
// Design (GB300):
// * A CTA (one per SM) owns one 64 (u) x 32 (v) tile of the grid for a work
//   item (a run of that tile's bin) and keeps the tile's accumulators in
//   registers, so each grid point is committed once per work item (vector
//   atomics, red.global).
// * Sixteen compute warps each own an 8 (u) x 16 (v) block; lane (lu, lv)
//   holds the points (lu, lv + 4 j), j = 0..3 ("slots" of 8 x 4 points), for
//   every polarisation.  Four slots per warp amortise each record's staged
//   visibility over up to 4 x 32 points.  (The lane layout is a compile-time
//   choice, kGridLanesU x kGridLanesV = 8 x 4 or 16 x 2; the text describes
//   the default.)
// * The work is bound by the gathers of kernel values from L2 (each a
//   4-row x 64-byte window of a table slice per slot) and by the FP32 pipe,
//   so the design keeps many gathers in flight and many warps issuing: 20
//   warps per SM (4 compute warps and one producer warp per scheduler, 96
//   registers per thread), each compute warp holding the kernel values of
//   the next R = 3 list entries in a ring of registers.
// * Four producer warps (one warpgroup) stage batches of 256 records into
//   shared memory: the record ids and index records are loaded for all rows
//   at once, the visibilities are copied straight into shared memory with
//   cp.async (or widened / weighted in registers for 16-bit or weighted
//   input), and every record is appended to the list of each compute warp
//   whose block its footprint meets, with the record's table offset for the
//   tile and the slots its rows meet (one 64-bit entry).  Compute warps
//   therefore only see records that touch them.
// * Hand-over through mbarriers: a compute warp waits only for the batch it
//   needs and releases it when done, so the sixteen compute warps run
//   independently; the producers wait until all of them have released a
//   buffer before refilling it.  Every wait is bounded: a wait that gives up
//   sets the plan's device status word and the kernel returns.
// * The producers pad every warp's list to a multiple of R and append R more
//   null entries (no loads, the all-zero visibility row), so the compute loop
//   has no tail tests: the kernel values of entry i + R are loaded into the
//   registers entry i has just used, and the last pass over a batch loads the
//   first entries of the next batch (the ring never drains between batches).
//   An entry loads the slots its record
//   meets and zeros for the others, and always updates all four slots (one
//   loop body, no per-entry jump: the code stays small at ring depth R).
// * Kernel values come from zero-padded slices (kGridPadC = 7 zero columns
//   and kGridPadR = 3 zero rows around each S x S slice, one compile-time
//   row stride per plan), so
//   lanes outside the footprint read zeros and slot addresses are immediate
//   offsets.
// * Per tap and polarisation the update is two packed FP32x2 FMAs (Blackwell
//   FFMA2) on the (re, im) accumulator pair:
//     acc += (K.re, K.re) (.) (V.re, V.im) + (K.im, K.im) (.) s (-V.im, V.re)
//   with s = -1 for the conjugate kernel (w < 0); the staged visibility is
//   the plain (weighted) value, the second operand is formed in registers.
// * Storage precision: the table element type is a template parameter
//   (complex FP32, or bfloat16 / float16 pairs widened to FP32 on load);
//   visibilities of any kind are widened to FP32 when staged; all
//   accumulation is FP32.  With an error grid the commit is compensated
//   (commit_compensated).
#pragma once

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kBlockU = kGridLanesU;                      // warp block: kBlockU (u) x kBlockV (v)
constexpr int kBlockV = 4 * kGridLanesV;
constexpr int kBlocksU = kGridTileU / kBlockU;            // blocks per tile row
constexpr int kComputeWarps = kBlocksU * (kGridTileV / kBlockV);
#ifndef GW_GRID_PRODUCER_WARPS
#define GW_GRID_PRODUCER_WARPS 4
#endif
constexpr int kProducerWarps = GW_GRID_PRODUCER_WARPS;
constexpr int kProducerThreads = kProducerWarps * 32;
constexpr int kThreads = (kComputeWarps + kProducerWarps) * 32;
constexpr int kBatch = 256;
constexpr int kPerLane = kBatch / kProducerThreads;   // rows staged by each producer thread
constexpr int kProducerBar = 1;                        // named barrier of the producer warps

// entry.y: record row in the batch (bits 0-8), conjugate kernel (bit 19),
// mask of the slots the record's rows meet (bits 20-23)
constexpr uint32_t kZeroRow = kBatch;   // staged visibility row that is always zero
constexpr uint32_t kConjBit = 1u << 19;
__device__ __forceinline__ gw_index_rec load_rec(const gw_index_rec* rec, uint32_t i) {
    int4 v = __ldg(reinterpret_cast<const int4*>(rec) + i);
    return *reinterpret_cast<gw_index_rec*>(&v);
}

// ---- mbarriers (shared memory, CTA scope) ----------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the completion of the barrier phase of the given parity; gives
// up after about two seconds (a batch hand-over takes microseconds).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}
__device__ __forceinline__ void producer_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kProducerBar), "n"(kProducerThreads) : "memory");
}

// ---- asynchronous global -> shared copies ----------------------------------
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
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

template <int R>
constexpr int list_cap() { return kBatch + 2 * R; }

template <int NPOL, int B, int R>
struct Smem {
    float2 v[B][kBatch + 1][NPOL];          // weighted visibilities; row kBatch = 0
    // per warp: list entries, padded to a multiple of R, then R null entries
    uint2 list[B][kComputeWarps][list_cap<R>()];
    int cnt[B][kComputeWarps];             // entries, padded to a multiple of R
    int tile[B];                           // tile of the batch; -1 = end of work
    int last[B];                           // batch ends its work item
    Item item;                             // producers: the current work item
    int done;                              // producers: no work item left
    unsigned long long full[B], empty[B];  // mbarriers
};

// Packed FMAs of one entry into slots J0..J1 (compile-time range); A = V,
// Bv = s (-V.im, V.re) (unused for a real kernel).
template <int NPOL, int J0, int J1, class TE>
__device__ __forceinline__ void slot_fma(float2 (&acc)[4][NPOL], const typename TE::T (&Kr)[4],
                                         const float2 (&A)[NPOL], const float2 (&Bv)[NPOL]) {
#pragma unroll
    for (int j = J0; j <= J1; ++j) {
        const float2 kc = TE::cvt(Kr[j]);   // 16-bit pairs are widened here, at their use
        const float2 kxx = make_float2(kc.x, kc.x);
        const float2 kyy = make_float2(kc.y, kc.y);
#pragma unroll
        for (int p = 0; p < NPOL; ++p) acc[j][p] = __ffma2_rn(kxx, A[p], acc[j][p]);
        if constexpr (!TE::kReal) {
#pragma unroll
            for (int p = 0; p < NPOL; ++p) acc[j][p] = __ffma2_rn(kyy, Bv[p], acc[j][p]);
        }
    }
}

// Staged visibility of an entry and the second FMA operand s (-V.im, V.re)
// (not formed for a real kernel).
template <int NPOL, bool REAL>
__device__ __forceinline__ void load_v(float2 (&A)[NPOL], float2 (&Bv)[NPOL],
                                       const float2 (*vs)[NPOL], uint32_t ey) {
    const float2* row = vs[ey & 0x1ff];
    if (NPOL % 2 == 0) {
#pragma unroll
        for (int p = 0; p < NPOL; p += 2) {
            const float4 q = *reinterpret_cast<const float4*>(row + p);
            A[p] = make_float2(q.x, q.y);
            A[p + 1] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int p = 0; p < NPOL; ++p) A[p] = row[p];
    }
    if constexpr (!REAL) {
        const float s = (ey & kConjBit) ? -1.f : 1.f;
#pragma unroll
        for (int p = 0; p < NPOL; ++p) Bv[p] = make_float2(-s * A[p].y, s * A[p].x);
    }
}

// Kernel values of one list entry, as stored: the slots in its mask, zero
// (all bits clear, +0 in every storage kind) for the others.
template <int SP, class TE>
__device__ __forceinline__ void load_masked(const typename TE::T* __restrict__ tab, const uint2 en,
                                            typename TE::T (&Kd)[4]) {
    using T = typename TE::T;
    const uint32_t m = en.y >> 20;
    const T* p_ = tab + (int)en.x;
    const T z{};
    Kd[0] = (m & 1u) ? __ldg(p_) : z;
    Kd[1] = (m & 2u) ? __ldg(p_ + kGridLanesV * SP) : z;
    Kd[2] = (m & 4u) ? __ldg(p_ + 2 * kGridLanesV * SP) : z;
    Kd[3] = (m & 8u) ? __ldg(p_ + 3 * kGridLanesV * SP) : z;
}

// Fills the ring with the first R entries of a list.
template <int SP, int R, class TE>
__device__ __forceinline__ void ring_fill(const uint2* lst, const typename TE::T* __restrict__ tab,
                                          typename TE::T (&K)[R][4], uint32_t (&ey)[R]) {
#pragma unroll
    for (int d = 0; d < R; ++d) {
        const uint2 en = lst[d];
        ey[d] = en.y;
        load_masked<SP, TE>(tab, en, K[d]);
    }
}

// One ring pass: the FMAs of the R entries in the ring, each followed by the
// loads of the entry R positions later, taken from `next`.  Every entry
// updates all four slots; the slots outside its mask add zeros (spare FMA
// issue, but one short loop body per ring position and no per-entry jump).
template <int NPOL, int SP, int R, class TE>
__device__ __forceinline__ void ring_pass(const uint2* next, const float2 (*vs)[NPOL],
                                          const typename TE::T* __restrict__ tab,
                                          typename TE::T (&K)[R][4], uint32_t (&ey)[R],
                                          float2 (&acc)[4][NPOL]) {
#pragma unroll
    for (int d = 0; d < R; ++d) {
        float2 A[NPOL], Bv[NPOL];
        load_v<NPOL, TE::kReal>(A, Bv, vs, ey[d]);
        slot_fma<NPOL, 0, 3, TE>(acc, K[d], A, Bv);
        const uint2 en = next[d];
        ey[d] = en.y;
        load_masked<SP, TE>(tab, en, K[d]);
    }
}

template <int NPOL, int SP, int TK, int B, int R>
__global__ void __launch_bounds__(kThreads, 1) k_grid(GridArgs a) {
    using TE = TabElem<TK>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<NPOL, B, R>& sm = *reinterpret_cast<Smem<NPOL, B, R>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int side = a.ntiles_u;
    const int hb = a.beta / 2;

    // one-time set-up: barriers, the zero visibility row
    if (threadIdx.x == 0) {
        for (int b = 0; b < B; ++b) {
            mbar_init(&sm.full[b], kProducerThreads);
            mbar_init(&sm.empty[b], kComputeWarps * 32);
        }
    }
    for (int t = threadIdx.x; t < B * NPOL; t += kThreads)
        sm.v[t / NPOL][kZeroRow][t % NPOL] = make_float2(0.f, 0.f);
    __syncthreads();

    if (warp >= kComputeWarps) {
#ifdef GW_GRID_SETMAXNREG
        asm volatile("setmaxnreg.dec.sync.aligned.u32 40;" ::: "memory");
#endif
        // ----------------------------------------------------------- producers
        const int pt = threadIdx.x - kComputeWarps * 32;   // 0 .. kProducerThreads - 1
        const int pw = pt >> 5;
        // items [i0, *item_count): a band of tile rows, or all of them
        const uint32_t i0 = a.item_first ? *a.item_first : 0u;
        const uint32_t nitems = *a.item_count - i0;
        // visibilities copied as they are: FP32 pairs without weights, with
        // the 16-byte alignment the 16-byte copies need (pairs of polarisations)
        const bool copy_vis = a.vis_kind == GW_C64 && a.weight == nullptr &&
                              (NPOL % 2 == 1 || reinterpret_cast<uintptr_t>(a.vis) % 16 == 0);
        uint32_t nbatch = 0;
        for (;;) {
            int b = 0, nb_total = 1;
            bool done = false;
            Item item{};
            for (;;) {   // batches of the current work item
                const int buf = nbatch % B;
                if (nbatch >= (uint32_t)B &&
                    !mbar_wait(&sm.empty[buf], ((nbatch / B) - 1) & 1)) {
                    if (lane == 0) atomicOr(a.queue + 1, 1u);
                    return;
                }
                if (pw == 0) {
                    if (b == 0 && lane == 0) {
                        const uint32_t it = atomicAdd(a.queue, 1u);
                        sm.done = it >= nitems;
                        if (it < nitems) sm.item = a.items[i0 + it];
                    }
                    if (lane < kComputeWarps) sm.cnt[buf][lane] = 0;
                }
                producer_sync();
                if (b == 0) {
                    done = sm.done != 0;
                    if (!done) item = sm.item;
                    nb_total = done ? 1 : (item.len + kBatch - 1) / kBatch;
                }
                if (!done) {
                    // with w-layers (w-stacking) a tile id is layer * layer_tiles + tile
                    const int ltile = a.layer_tiles ? item.tile % a.layer_tiles : item.tile;
                    const int tu0 = (ltile % side) * kGridTileU;
                    const int tv0 = (ltile / side) * kGridTileV;
                    const int b0 = b * kBatch;
                    const int nb = min(kBatch, item.len - b0);
                    // all ids, then all index records of this thread's rows in flight
                    uint32_t ids[kPerLane];
                    gw_index_rec rcs[kPerLane];
#pragma unroll
                    for (int k = 0; k < kPerLane; ++k) {
                        const int r = k * kProducerThreads + pt;
                        ids[k] = r < nb ? __ldg(a.entries + item.start + b0 + r) : 0u;
                    }
#pragma unroll
                    for (int k = 0; k < kPerLane; ++k) {
                        const int r = k * kProducerThreads + pt;
                        if (r < nb) rcs[k] = load_rec(a.rec, ids[k]);
                    }
#pragma unroll
                    for (int k = 0; k < kPerLane; ++k) {
                        const int r = k * kProducerThreads + pt;
                        if (r >= nb) break;
                        const uint32_t id = ids[k];
                        const gw_index_rec rc = rcs[k];
                        if (copy_vis) {
                            const float2* src = reinterpret_cast<const float2*>(a.vis) +
                                                (int64_t)id * NPOL;
                            if (NPOL % 2 == 0) {
#pragma unroll
                                for (int p = 0; p < NPOL; p += 2)
                                    cp_async16(&sm.v[buf][r][p], src + p);
                            } else {
#pragma unroll
                                for (int p = 0; p < NPOL; ++p) cp_async8(&sm.v[buf][r][p], src + p);
                            }
                        } else {
#pragma unroll
                            for (int p = 0; p < NPOL; ++p) {
                                float2 v = load_vis(a.vis, a.vis_kind, (int64_t)id * NPOL + p);
                                if (a.weight) {
                                    const float w = __ldg(a.weight + (int64_t)id * NPOL + p);
                                    v.x *= w;
                                    v.y *= w;
                                }
                                sm.v[buf][r][p] = v;
                            }
                        }
                        // w-stacking records carry their layer in `plane`; the
                        // kernel is the plan's single (w = 0) plane
                        const int plane = (a.layer_tiles && !a.plane_groups) ? 0 : rc.plane;
                        const int S = __ldg(a.support + plane), h = S >> 1;
                        const int64_t slice = __ldg(a.pplane_off + plane) +
                                              ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) *
                                                  (int64_t)(S + 2 * kGridPadR) * SP;
                        // padded index of the tile origin relative to this record
                        const int base = (int)slice + (tv0 - rc.kv + h + kGridPadR) * SP +
                                         (tu0 - rc.ku + h + kGridPadC);
                        const uint32_t conj = (rc.flags & GW_FLAG_CONJ) ? kConjBit : 0u;
                        // footprint relative to the tile: [ulo, uhi] x [vlo, vhi]
                        const int ulo = rc.ku - h - tu0, uhi = rc.ku + h - tu0;
                        const int vlo = rc.kv - h - tv0, vhi = rc.kv + h - tv0;
                        const int cu0 = max(0, ulo) / kBlockU, cu1 = min(kGridTileU - 1, uhi) / kBlockU;
                        const int cv0 = max(0, vlo) / kBlockV, cv1 = min(kGridTileV - 1, vhi) / kBlockV;
                        for (int cv = cv0; cv <= cv1; ++cv) {
                            const int j0 = max(0, vlo - kBlockV * cv) / kGridLanesV;
                            const int j1 = min(kBlockV - 1, vhi - kBlockV * cv) / kGridLanesV;
                            const uint32_t mask = ((2u << j1) - 1u) & ~((1u << j0) - 1u);
                            const uint2 e = make_uint2((uint32_t)base,
                                                       (uint32_t)r | (mask << 20) | conj);
                            for (int cu = cu0; cu <= cu1; ++cu) {
                                const int w = cv * kBlocksU + cu;
#ifdef GW_DEBUG_BOUNDS
                                // the entry's loads: slots j0..j1 of the warp's block
                                const int64_t lo = (int64_t)base + (int64_t)(kBlockV * cv + kGridLanesV * j0) * SP +
                                                   kBlockU * cu;
                                const int64_t hi = (int64_t)base +
                                                   (int64_t)(kBlockV * cv + kGridLanesV * j1 + kGridLanesV - 1) * SP +
                                                   kBlockU * cu + kBlockU - 1;
                                if (!gw_in_bounds(a.ptable_elems == 0 || (lo >= 0 && hi < a.ptable_elems),
                                                  a.queue + 1))
                                    continue;
#endif
                                const int pos = atomicAdd(&sm.cnt[buf][w], 1);
                                if (gw_in_bounds(pos < kBatch, a.queue + 1)) sm.list[buf][w][pos] = e;
                            }
                        }
                    }
                    if (copy_vis) cp_async_wait_all();
                }
                producer_sync();   // all rows staged, all list appends done
                if (pw == 0) {
                    // pad every warp's list to a multiple of R and put R null
                    // entries (no slots loaded, the zero visibility row) after it
                    if (lane < kComputeWarps) {
                        const int w = lane;
                        const int nf = sm.cnt[buf][w];
                        const int nfp = (nf + R - 1) / R * R;
                        const uint2 z = make_uint2(0u, kZeroRow);
                        for (int k = nf; k < nfp + R; ++k) sm.list[buf][w][k] = z;
                        sm.cnt[buf][w] = nfp;
                    }
                    if (lane == 0) {
                        sm.tile[buf] = done ? -1 : item.tile;
                        sm.last[buf] = done ? 1 : (b == nb_total - 1);
                    }
                    __syncwarp();
                }
                mbar_arrive(&sm.full[buf]);  // batch ready (every producer thread)
                ++nbatch;
                if (++b == nb_total) break;
            }
            if (done) break;
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
#ifdef GW_GRID_SETMAXNREG
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(GW_GRID_SETMAXNREG) : "memory");
#endif
    const int bu = (warp % kBlocksU) * kBlockU, bv = (warp / kBlocksU) * kBlockV;
    const int lu = lane % kGridLanesU, lv = lane / kGridLanesU;
    const typename TE::T* __restrict__ tab =
        reinterpret_cast<const typename TE::T*>(a.ptable) + (bv + lv) * SP + bu + lu;
    const int N = a.N;
    float2 acc[4][NPOL];   // (re, im)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int p = 0; p < NPOL; ++p) acc[j][p] = make_float2(0.f, 0.f);
    // kernel-value ring, in the table's storage kind; finite values only
    // (zero, then table values), so the null entries' zero visibility row
    // contributes exact zeros
    typename TE::T K[R][4];
    uint32_t ey[R];
#pragma unroll
    for (int d = 0; d < R; ++d)
#pragma unroll
        for (int j = 0; j < 4; ++j) K[d][j] = typename TE::T{};

    // The ring runs across batches: the last pass over a batch's list loads
    // the first R entries of the next batch, so no batch starts with an empty
    // ring.  Lists are padded to a multiple of R and followed by R null
    // entries (the end-of-work batch has only those).
    if (!mbar_wait(&sm.full[0], 0)) {
        if (lane == 0) atomicOr(a.queue + 1, 1u);
        return;
    }
    ring_fill<SP, R, TE>(sm.list[0][warp], tab, K, ey);
    uint32_t nbatch = 0;
    for (;;) {
        const int buf = nbatch % B;
        const int tile = sm.tile[buf];
        if (tile < 0) break;
        const int last = sm.last[buf];
        const int n = sm.cnt[buf][warp];
        const uint2* lst = sm.list[buf][warp];
        const int nbuf = (nbatch + 1) % B;
        const uint2* nlst = sm.list[nbuf][warp];
        for (int i = 0;; i += R) {
            const bool tail = i + R >= n;
            if (tail && !mbar_wait(&sm.full[nbuf], ((nbatch + 1) / B) & 1)) {
                if (lane == 0) atomicOr(a.queue + 1, 1u);
                return;
            }
            if (n == 0) {   // nothing of this batch for this warp
                ring_fill<SP, R, TE>(nlst, tab, K, ey);
                break;
            }
            ring_pass<NPOL, SP, R, TE>(tail ? nlst : lst + i + R, sm.v[buf], tab, K, ey, acc);
            if (tail) break;
        }
        mbar_arrive(&sm.empty[buf]);  // buffer free (every lane, after its reads)
        ++nbatch;
        if (last) {
            // commit the tile's accumulators of this work item
            const int ltile = a.layer_tiles ? tile % a.layer_tiles : tile;
            float2* const gbase = a.grid + (a.layer_tiles ? (int64_t)(tile / a.layer_tiles) *
                                                                 a.layer_stride : 0);
            const int u = (ltile % a.ntiles_u) * kGridTileU + bu + lu;
            const int v0 = (ltile / a.ntiles_u) * kGridTileV + bv + lv;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int v = v0 + kGridLanesV * j;
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
    }
}

template <int NPOL, int SP, int TK, int B, int R>
void launch_v(const GridArgs& a, int num_sms, cudaStream_t s) {
    const size_t smem = sizeof(Smem<NPOL, B, R>);
    cudaFuncSetAttribute(k_grid<NPOL, SP, TK, B, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid<NPOL, SP, TK, B, R>, kThreads,
                                                  smem);
    if (per_sm < 1) per_sm = 1;
    k_grid<NPOL, SP, TK, B, R><<<num_sms * per_sm, kThreads, smem, s>>>(a);
    note_launch();
}

// GW_GRID_BUFS staging buffers of 256 records and a ring of GW_GRID_RING
// kernel-value register sets per compute warp (measured on the 4-pol
// w-projection batch: 16 compute warps with ring 3 beat 8 compute warps with
// rings of 2-10 entries at 168 registers).
#ifndef GW_GRID_RING
#define GW_GRID_RING 3
#endif
#ifndef GW_GRID_BUFS
#define GW_GRID_BUFS 4
#endif
template <int NPOL, int SP, int TK>
void launch_sp(const GridArgs& a, int num_sms, cudaStream_t s) {
    launch_v<NPOL, SP, TK, GW_GRID_BUFS, GW_GRID_RING>(a, num_sms, s);
}

template <int NPOL, int TK>
void launch_t(const GridArgs& a, int num_sms, cudaStream_t s) {
    switch (a.pad_stride) {
#if GW_GRID_LANES_U == 16
        case 32: launch_sp<NPOL, 32, TK>(a, num_sms, s); break;
        case 48: launch_sp<NPOL, 48, TK>(a, num_sms, s); break;
        case 64: launch_sp<NPOL, 64, TK>(a, num_sms, s); break;
        case 96: launch_sp<NPOL, 96, TK>(a, num_sms, s); break;
        case 160: launch_sp<NPOL, 160, TK>(a, num_sms, s); break;
        default: launch_sp<NPOL, 288, TK>(a, num_sms, s); break;
#else
        case 24: launch_sp<NPOL, 24, TK>(a, num_sms, s); break;
        case 32: launch_sp<NPOL, 32, TK>(a, num_sms, s); break;
        case 48: launch_sp<NPOL, 48, TK>(a, num_sms, s); break;
        case 80: launch_sp<NPOL, 80, TK>(a, num_sms, s); break;
        case 144: launch_sp<NPOL, 144, TK>(a, num_sms, s); break;
        default: launch_sp<NPOL, 272, TK>(a, num_sms, s); break;
#endif
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
