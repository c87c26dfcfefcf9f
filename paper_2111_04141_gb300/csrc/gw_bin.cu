// Device binner: groups visibility ids by grid tile.
//
// The thesis orders records by their position on the NN grid ("SS" mode,
// Section 3.3.5) because record order controls commit traffic.  Here the
// equivalent is a bin per grid tile (2^su x 2^sv pixels):
//   footprint mode: a record is listed in every tile its S_p x S_p footprint
//                   touches (the gridder owns a tile and needs all of them);
//   centre mode:    a record is listed once, in the tile of its pixel (the
//                   degridder reads a record's whole footprint).
// Steps: histogram (atomics; per-CTA shared histograms when the tile count
// allows) -> exclusive scan -> scatter (atomic cursors),
// then the footprint bins are cut into work items of at most item_max
// entries.  Order within a bin is unspecified.
#include "gw_internal.cuh"

namespace gw {

namespace {

struct TileRange {
    int tu0, tu1, tv0, tv1;
};

__device__ __forceinline__ TileRange tile_range(const gw_index_rec& r, const BinGeom& g, int P,
                                                int smin, int smax) {
    TileRange t;
    if (g.mode == 1) {
        t.tu0 = t.tu1 = r.ku >> g.su;
        t.tv0 = t.tv1 = r.kv >> g.sv;
    } else {
        const int h = plane_support(r.plane, P, smin, smax) / 2;
        t.tu0 = (r.ku - h) >> g.su;
        t.tu1 = (r.ku + h) >> g.su;
        t.tv0 = (r.kv - h) >> g.sv;
        t.tv1 = (r.kv + h) >> g.sv;
    }
    return t;
}

__device__ __forceinline__ gw_index_rec load_rec(const gw_index_rec* rec, int64_t i) {
    int4 v = __ldg(reinterpret_cast<const int4*>(rec) + i);
    return *reinterpret_cast<gw_index_rec*>(&v);
}

__global__ void k_count(const gw_index_rec* __restrict__ rec, int64_t nvis, DevCount dc, BinGeom g,
                        int P, int smin, int smax, uint32_t* __restrict__ count,
                        unsigned long long* __restrict__ work) {
    nvis = dc.clamp(nvis);
    unsigned long long n_valid = 0, n_taps = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvis;
         i += (int64_t)gridDim.x * blockDim.x) {
        const gw_index_rec r = load_rec(rec, i);
        if (!(r.flags & GW_FLAG_VALID)) continue;
        const int S = plane_support(r.plane, P, smin, smax);
        ++n_valid;
        n_taps += (unsigned long long)(S * S);
        const TileRange t = tile_range(r, g, P, smin, smax);
        const int lbase = g.layer_tiles ? (r.plane / g.group_planes) * g.layer_tiles : 0;
        for (int tv = t.tv0; tv <= t.tv1; ++tv)
            for (int tu = t.tu0; tu <= t.tu1; ++tu)
                atomicAdd(count + lbase + tv * g.ntu + tu, 1u);
    }
    for (int d = 16; d > 0; d >>= 1) {
        n_valid += __shfl_down_sync(0xffffffffu, n_valid, d);
        n_taps += __shfl_down_sync(0xffffffffu, n_taps, d);
    }
    if ((threadIdx.x & 31) == 0 && n_valid) {
        atomicAdd(work, n_valid);
        atomicAdd(work + 1, n_taps);
    }
}

// Exclusive scans of count[] -> offsets[], and of ceil(count / item_max) ->
// item_off[], in one block.  n may exceed the block size; each thread scans
// a contiguous run, then the run totals are scanned across the block.
__global__ void k_scan(const uint32_t* __restrict__ count, int n, int item_max,
                       uint32_t* __restrict__ offsets, uint32_t* __restrict__ item_off,
                       uint32_t* __restrict__ cursor) {
    __shared__ uint32_t s_a[1024];
    __shared__ uint32_t s_b[1024];
    const int tid = threadIdx.x;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    uint32_t sa = 0, sb = 0;
    for (int i = lo; i < hi; ++i) {
        const uint32_t c = count[i];
        sa += c;
        sb += (c + item_max - 1) / item_max;
    }
    s_a[tid] = sa;
    s_b[tid] = sb;
    __syncthreads();
    // Hillis-Steele inclusive scan over the run totals
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {
        uint32_t xa = 0, xb = 0;
        if (tid >= d) {
            xa = s_a[tid - d];
            xb = s_b[tid - d];
        }
        __syncthreads();
        s_a[tid] += xa;
        s_b[tid] += xb;
        __syncthreads();
    }
    uint32_t ra = s_a[tid] - sa, rb = s_b[tid] - sb;
    for (int i = lo; i < hi; ++i) {
        const uint32_t c = count[i];
        offsets[i] = ra;
        item_off[i] = rb;
        cursor[i] = 0;
        ra += c;
        rb += (c + item_max - 1) / item_max;
    }
    if (tid == blockDim.x - 1) {
        offsets[n] = s_a[tid];
        item_off[n] = s_b[tid];
    }
}

// Segmented scans for many bins: segments of kScanSeg bins, one CTA each.
// Pass 0 writes each segment's totals (bins and work items); k_scan_top scans
// the totals in one CTA; pass 1 writes offsets, item offsets and zeroed
// cursors with the segment's base.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanSeg = kScanThreads * kScanPer;
constexpr int kScanSingleMax = 65536;

__device__ __forceinline__ void block_excl_scan2(uint32_t& a, uint32_t& b, uint32_t* sa,
                                                 uint32_t* sb) {
    // exclusive scan of (a, b) over the CTA (kScanThreads threads)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t ia = a, ib = b;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t xa = __shfl_up_sync(0xffffffffu, ia, d);
        const uint32_t xb = __shfl_up_sync(0xffffffffu, ib, d);
        if (lane >= d) { ia += xa; ib += xb; }
    }
    if (lane == 31) { sa[warp] = ia; sb[warp] = ib; }
    __syncthreads();
    if (warp == 0) {
        uint32_t wa = sa[lane], wb = sb[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t xa = __shfl_up_sync(0xffffffffu, wa, d);
            const uint32_t xb = __shfl_up_sync(0xffffffffu, wb, d);
            if (lane >= d) { wa += xa; wb += xb; }
        }
        sa[lane] = wa;
        sb[lane] = wb;
    }
    __syncthreads();
    const uint32_t ba = warp ? sa[warp - 1] : 0u, bb = warp ? sb[warp - 1] : 0u;
    a = ba + ia - a;
    b = bb + ib - b;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_seg(
    const uint32_t* __restrict__ count, int n, int item_max, int pass,
    uint32_t* __restrict__ seg_tot, uint32_t* __restrict__ offsets,
    uint32_t* __restrict__ item_off, uint32_t* __restrict__ cursor) {
    __shared__ uint32_t sa[32], sb[32];
    const int64_t i0 = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanPer;
    uint32_t c[kScanPer];
    uint32_t ta = 0, tb = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        c[k] = i0 + k < n ? count[i0 + k] : 0u;
        ta += c[k];
        tb += (c[k] + item_max - 1) / item_max;
    }
    uint32_t ea = ta, eb = tb;
    block_excl_scan2(ea, eb, sa, sb);
    if (pass == 0) {
        if (threadIdx.x == kScanThreads - 1) {
            seg_tot[2 * blockIdx.x] = ea + ta;
            seg_tot[2 * blockIdx.x + 1] = eb + tb;
        }
        return;
    }
    uint32_t ra = seg_tot[2 * blockIdx.x] + ea, rb = seg_tot[2 * blockIdx.x + 1] + eb;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (i0 + k < n) {
            offsets[i0 + k] = ra;
            item_off[i0 + k] = rb;
            cursor[i0 + k] = 0;
        }
        ra += c[k];
        rb += (c[k] + item_max - 1) / item_max;
    }
}

// Exclusive scan of the segment totals in place (one CTA, nseg <= 32 * 1024);
// writes the grand totals to offsets[n] and item_off[n].
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t* __restrict__ seg_tot, int nseg,
                                                           int n, uint32_t* __restrict__ offsets,
                                                           uint32_t* __restrict__ item_off) {
    __shared__ uint32_t sa[32], sb[32];
    const int per = (nseg + kScanThreads - 1) / kScanThreads;
    const int lo = min(nseg, (int)threadIdx.x * per), hi = min(nseg, lo + per);
    uint32_t ta = 0, tb = 0;
    for (int i = lo; i < hi; ++i) {
        ta += seg_tot[2 * i];
        tb += seg_tot[2 * i + 1];
    }
    uint32_t ea = ta, eb = tb;
    block_excl_scan2(ea, eb, sa, sb);
    for (int i = lo; i < hi; ++i) {
        const uint32_t xa = seg_tot[2 * i], xb = seg_tot[2 * i + 1];
        seg_tot[2 * i] = ea;
        seg_tot[2 * i + 1] = eb;
        ea += xa;
        eb += xb;
    }
    if (threadIdx.x == kScanThreads - 1) {
        offsets[n] = ea;
        item_off[n] = eb;
    }
}

__global__ void k_scatter(const gw_index_rec* __restrict__ rec, int64_t nvis, DevCount dc,
                          BinGeom g, int P, int smin, int smax,
                          const uint32_t* __restrict__ offsets, uint32_t* __restrict__ cursor,
                          uint32_t* __restrict__ entries) {
    nvis = dc.clamp(nvis);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvis;
         i += (int64_t)gridDim.x * blockDim.x) {
        const gw_index_rec r = load_rec(rec, i);
        if (!(r.flags & GW_FLAG_VALID)) continue;
        const TileRange t = tile_range(r, g, P, smin, smax);
        const int lbase = g.layer_tiles ? (r.plane / g.group_planes) * g.layer_tiles : 0;
        for (int tv = t.tv0; tv <= t.tv1; ++tv)
            for (int tu = t.tu0; tu <= t.tu1; ++tu) {
                const int tile = lbase + tv * g.ntu + tu;
                const uint32_t pos = atomicAdd(cursor + tile, 1u);
                entries[offsets[tile] + pos] = (uint32_t)i;
            }
    }
}

// Shared-memory variants (ntiles small enough for a per-CTA histogram): a
// CTA takes a contiguous chunk of records and counts its (record, tile)
// pairs with shared-memory atomics; only the non-zero bins reach global
// memory, one atomic each.  The scatter recounts its chunk, reserves one run
// per (CTA, tile) in the tile's bin with a single global atomic, and places
// the entries with shared-memory cursors that start at the run bases.
constexpr int kBinSmThreads = 512;
constexpr int kBinSmTilesMax = 49152;     // 192 KB of u32 counters

__global__ void __launch_bounds__(kBinSmThreads) k_count_sm(
    const gw_index_rec* __restrict__ rec, int64_t nvis, DevCount dc, BinGeom g, int P, int smin,
    int smax, int ntiles, uint32_t* __restrict__ count, unsigned long long* __restrict__ work) {
    extern __shared__ uint32_t hist[];
    nvis = dc.clamp(nvis);
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const int64_t chunk = (nvis + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = blockIdx.x * chunk, c1 = min(nvis, c0 + chunk);
    unsigned long long n_valid = 0, n_taps = 0;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const gw_index_rec r = load_rec(rec, i);
        if (!(r.flags & GW_FLAG_VALID)) continue;
        const int S = plane_support(r.plane, P, smin, smax);
        ++n_valid;
        n_taps += (unsigned long long)(S * S);
        const TileRange t = tile_range(r, g, P, smin, smax);
        const int lbase = g.layer_tiles ? (r.plane / g.group_planes) * g.layer_tiles : 0;
        for (int tv = t.tv0; tv <= t.tv1; ++tv)
            for (int tu = t.tu0; tu <= t.tu1; ++tu) atomicAdd(hist + lbase + tv * g.ntu + tu, 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        if (hist[t]) atomicAdd(count + t, hist[t]);
    for (int d = 16; d > 0; d >>= 1) {
        n_valid += __shfl_down_sync(0xffffffffu, n_valid, d);
        n_taps += __shfl_down_sync(0xffffffffu, n_taps, d);
    }
    if ((threadIdx.x & 31) == 0 && n_valid) {
        atomicAdd(work, n_valid);
        atomicAdd(work + 1, n_taps);
    }
}

__global__ void __launch_bounds__(kBinSmThreads) k_scatter_sm(
    const gw_index_rec* __restrict__ rec, int64_t nvis, DevCount dc, BinGeom g, int P, int smin,
    int smax, int ntiles, const uint32_t* __restrict__ offsets, uint32_t* __restrict__ cursor,
    uint32_t* __restrict__ entries) {
    extern __shared__ uint32_t hist[];
    nvis = dc.clamp(nvis);
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const int64_t chunk = (nvis + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = blockIdx.x * chunk, c1 = min(nvis, c0 + chunk);
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const gw_index_rec r = load_rec(rec, i);
        if (!(r.flags & GW_FLAG_VALID)) continue;
        const TileRange t = tile_range(r, g, P, smin, smax);
        const int lbase = g.layer_tiles ? (r.plane / g.group_planes) * g.layer_tiles : 0;
        for (int tv = t.tv0; tv <= t.tv1; ++tv)
            for (int tu = t.tu0; tu <= t.tu1; ++tu) atomicAdd(hist + lbase + tv * g.ntu + tu, 1u);
    }
    __syncthreads();
    // this CTA's run in each bin: absolute position of its first entry
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t c = hist[t];
        if (c) hist[t] = offsets[t] + atomicAdd(cursor + t, c);
    }
    __syncthreads();
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const gw_index_rec r = load_rec(rec, i);
        if (!(r.flags & GW_FLAG_VALID)) continue;
        const TileRange t = tile_range(r, g, P, smin, smax);
        const int lbase = g.layer_tiles ? (r.plane / g.group_planes) * g.layer_tiles : 0;
        for (int tv = t.tv0; tv <= t.tv1; ++tv)
            for (int tu = t.tu0; tu <= t.tu1; ++tu) {
                const uint32_t pos = atomicAdd(hist + lbase + tv * g.ntu + tu, 1u);
                entries[pos] = (uint32_t)i;
            }
    }
}

__global__ void k_items(const uint32_t* __restrict__ count, const uint32_t* __restrict__ offsets,
                        const uint32_t* __restrict__ item_off, int ntiles, int item_max,
                        Item* __restrict__ items) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        const uint32_t c = count[t];
        uint32_t o = item_off[t];
        for (uint32_t s = 0; s < c; s += (uint32_t)item_max, ++o) {
            Item it;
            it.tile = t;
            it.start = (int32_t)(offsets[t] + s);
            it.len = (int32_t)min((uint32_t)item_max, c - s);
            it.pad = 0;
            items[o] = it;
        }
    }
}

}  // namespace

void launch_bin(const gw_index_rec* rec, int64_t nvis, const BinGeom& g, int P, int smin, int smax,
                Scratch& sc, cudaStream_t s, DevCount dc) {
    const int ntiles = g.ntu * g.ntv * (g.layer_tiles ? g.nlayers : 1);
    cudaMemsetAsync(sc.count, 0, sizeof(uint32_t) * ntiles, s);
    // per-CTA shared histograms when the bins fit and every CTA has at
    // least ntiles records (zeroing and flushing its histogram stays a small
    // part of its work); small inputs keep the global-atomic kernels, which
    // also leave the GPU to concurrent work on other streams
    int sm_blocks = 0;
    const size_t hsm = sizeof(uint32_t) * (size_t)ntiles;
    if (ntiles <= kBinSmTilesMax && nvis >= 2LL * ntiles) {
        int dev = 0, nsm = 0, c_sm = 0, s_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_count_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        cudaFuncSetAttribute(k_scatter_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c_sm, k_count_sm, kBinSmThreads, hsm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s_sm, k_scatter_sm, kBinSmThreads, hsm);
        sm_blocks = (int)std::min<int64_t>((int64_t)std::min(c_sm, s_sm) * nsm,
                                           nvis / ntiles);
    }
    const int threads = 256;
    int64_t blocks = (nvis + threads - 1) / threads;
    if (blocks > current_sm_count() * 8) blocks = current_sm_count() * 8;
    if (blocks < 1) blocks = 1;
    if (nvis > 0) {
        if (sm_blocks > 0)
            k_count_sm<<<sm_blocks, kBinSmThreads, hsm, s>>>(rec, nvis, dc, g, P, smin, smax, ntiles,
                                                             sc.count, sc.work);
        else
            k_count<<<(unsigned)blocks, threads, 0, s>>>(rec, nvis, dc, g, P, smin, smax, sc.count,
                                                         sc.work);
        note_launch();
    }
    // one CTA scans up to 64 bins per thread quickly; beyond that, segments
    if (ntiles <= kScanSingleMax || !sc.scan_tmp || ntiles > sc.scan_tmp_bins) {
        k_scan<<<1, 1024, 0, s>>>(sc.count, ntiles, g.item_max, sc.offsets, sc.item_off,
                                  sc.cursor);
        note_launch();
    } else {
        const int nseg = (ntiles + kScanSeg - 1) / kScanSeg;
        k_scan_seg<<<nseg, kScanThreads, 0, s>>>(sc.count, ntiles, g.item_max, 0, sc.scan_tmp,
                                                 sc.offsets, sc.item_off, sc.cursor);
        k_scan_top<<<1, kScanThreads, 0, s>>>(sc.scan_tmp, nseg, ntiles, sc.offsets, sc.item_off);
        k_scan_seg<<<nseg, kScanThreads, 0, s>>>(sc.count, ntiles, g.item_max, 1, sc.scan_tmp,
                                                 sc.offsets, sc.item_off, sc.cursor);
        note_launch(3);
    }
    if (nvis > 0) {
        if (sm_blocks > 0)
            k_scatter_sm<<<sm_blocks, kBinSmThreads, hsm, s>>>(rec, nvis, dc, g, P, smin, smax,
                                                               ntiles, sc.offsets, sc.cursor,
                                                               sc.entries);
        else
            k_scatter<<<(unsigned)blocks, threads, 0, s>>>(rec, nvis, dc, g, P, smin, smax,
                                                           sc.offsets, sc.cursor, sc.entries);
        note_launch();
    }
    if (sc.items) {   // work items (the allocation-free degrid path has none)
        const int tb = (ntiles + 255) / 256;
        k_items<<<tb, 256, 0, s>>>(sc.count, sc.offsets, sc.item_off, ntiles, g.item_max, sc.items);
        note_launch();
    }
}

cudaError_t preload_bin_kernels() {
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, k_count);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_count_sm);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_scan);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_scatter);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_scatter_sm);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_items);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_scan_seg);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, k_scan_top);
    return e;
}

int64_t scan_tmp_words(int64_t ntiles) { return 2 * ((ntiles + kScanSeg - 1) / kScanSeg) + 2; }

}  // namespace gw
