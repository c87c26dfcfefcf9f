// Full compression (Section 3.3.5, "Full Compression"): visibility records
// that fall on the same pixel of the virtual NN grid -- here the same
// (k_u, k_v, o_u, o_v) on the beta-oversampled grid, the same w-plane and
// the same sign of w, i.e. the same kernel at the same place -- are added
// before gridding.  Gridding is linear, so the result is unchanged up to
// FP32 rounding while the gridder sees fewer records.
//
// GB300 form: one pass of open-addressing hash inserts (64-bit keys,
// atomicCAS, linear probing in a table at most half full) that also sums
// the weighted visibilities of each key with vector atomics, then one pass
// that compacts the occupied slots into records + visibilities and clears
// the table for the next chunk.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr unsigned long long kEmpty = ~0ULL;

// Key layout (59 bits): kv | ku << 15 | (ov + b/2) << 30 | (ou + b/2) << 38 |
// conj << 46 | plane << 47  (N <= 32768, beta <= 256, P <= 4096).
__device__ __forceinline__ unsigned long long make_key(const gw_index_rec& r, int hb) {
    return (unsigned long long)r.kv | ((unsigned long long)r.ku << 15) |
           ((unsigned long long)(r.ov + hb) << 30) | ((unsigned long long)(r.ou + hb) << 38) |
           ((unsigned long long)((r.flags & GW_FLAG_CONJ) ? 1 : 0) << 46) |
           ((unsigned long long)r.plane << 47);
}

__device__ __forceinline__ gw_index_rec key_rec(unsigned long long k, int hb) {
    gw_index_rec r;
    r.kv = (int32_t)(k & 0x7fff);
    r.ku = (int32_t)((k >> 15) & 0x7fff);
    r.ov = (int16_t)((int)((k >> 30) & 0xff) - hb);
    r.ou = (int16_t)((int)((k >> 38) & 0xff) - hb);
    const bool conj = (k >> 46) & 1;
    r.plane = (int16_t)(k >> 47);
    r.flags = (uint16_t)(GW_FLAG_VALID | (conj ? GW_FLAG_CONJ : 0u));
    return r;
}

// 64-bit finaliser of the SplitMix64 generator (Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void k_hash_insert(const gw_index_rec* __restrict__ rec, int64_t nvis,
                              const void* __restrict__ vis, int vis_kind,
                              const float* __restrict__ weight, int npol, int hb,
                              unsigned long long* __restrict__ keys, float2* __restrict__ acc,
                              unsigned long long mask, unsigned long long* __restrict__ n_in) {
    unsigned long long mine = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvis;
         i += (int64_t)gridDim.x * blockDim.x) {
        int4 rv = __ldg(reinterpret_cast<const int4*>(rec) + i);
        const gw_index_rec r = *reinterpret_cast<gw_index_rec*>(&rv);
        if (!(r.flags & GW_FLAG_VALID)) continue;
        ++mine;
        const unsigned long long key = make_key(r, hb);
        unsigned long long h = mix64(key) & mask;
        // at most half the table is occupied, so an empty slot is found in
        // far fewer than mask + 1 probes; the bound only guards the loop
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(keys + h, kEmpty, key);
            if (prev == kEmpty || prev == key) break;
            h = (h + 1) & mask;
        }
        for (int p = 0; p < npol; ++p) {
            float2 v = load_vis(vis, vis_kind, i * npol + p);
            if (weight) {
                const float w = __ldg(weight + i * npol + p);
                v.x *= w;
                v.y *= w;
            }
            atomicAdd(acc + h * npol + p, v);
        }
    }
    for (int d = 16; d > 0; d >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, d);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(n_in, mine);
}

__global__ void k_compact(unsigned long long* __restrict__ keys, float2* __restrict__ acc,
                          int64_t cap, int npol, int hb, gw_index_rec* __restrict__ rec_out,
                          float2* __restrict__ vis_out, unsigned long long* __restrict__ count,
                          unsigned long long* __restrict__ total) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap;
         s += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[s];
        if (k == kEmpty) continue;
        const unsigned long long pos = atomicAdd(count, 1ULL);
        atomicAdd(total, 1ULL);
        const gw_index_rec r = key_rec(k, hb);
        reinterpret_cast<int4*>(rec_out)[pos] = *reinterpret_cast<const int4*>(&r);
        for (int p = 0; p < npol; ++p) {
            vis_out[pos * npol + p] = acc[s * npol + p];
            acc[s * npol + p] = make_float2(0.f, 0.f);
        }
        keys[s] = kEmpty;                     // ready for the next chunk
    }
}

unsigned blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > current_sm_count() * 16) b = current_sm_count() * 16;
    return (unsigned)std::max<int64_t>(b, 1);
}

}  // namespace

void launch_compress(const gw_index_rec* rec, int64_t nvis, const void* vis, int vis_kind,
                     const float* weight, int npol, int beta, CompressScratch& cs,
                     cudaStream_t s) {
    cudaMemsetAsync(cs.count, 0, sizeof(unsigned long long), s);
    if (nvis > 0) {
        k_hash_insert<<<blocks_for(nvis), 256, 0, s>>>(rec, nvis, vis, vis_kind, weight, npol,
                                                       beta / 2, cs.keys, cs.acc,
                                                       (unsigned long long)(cs.cap - 1),
                                                       cs.n_in);
        note_launch();
    }
    k_compact<<<blocks_for(cs.cap), 256, 0, s>>>(cs.keys, cs.acc, cs.cap, npol, beta / 2,
                                                 cs.rec, cs.vis, cs.count, cs.total);
    note_launch();
}

void clear_compress_table(CompressScratch& cs, int npol, cudaStream_t s) {
    cudaMemsetAsync(cs.keys, 0xff, sizeof(unsigned long long) * cs.cap, s);
    cudaMemsetAsync(cs.acc, 0, sizeof(float2) * cs.cap * npol, s);
}

}  // namespace gw
