// Index stage: uvw (metres) x frequency -> pixel, oversampled offset, w-plane.
//
// This is the pre-processing the thesis moves out of the gridder
// (Section 3.3.5): each record's uv coordinate becomes integer indices of
// the beta-oversampled grid (nearest neighbour, Section 2.3.6), and records
// whose footprint leaves the grid are dropped (Bounded Records Assumption,
// Section 2.3.1).  Every floating-point step is an explicitly rounded FP64
// intrinsic, so no multiply-add is ever fused and the result is bit-exact
// with any IEEE-754 implementation of the same sequence.
//
// FP64 division and square root are slow on this GPU, so the sequence has
// one division per channel (the factor f / c0, shared by u, v and w) and
// none per visibility; the w-plane (nearest in sqrt|w|, ties up) is a count
// of precomputed thresholds T_j = ((j - 1/2)/(P - 1))^2 w_max, found by
// binary search.  Each CTA builds both small tables in shared memory.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kChanCache = 1024;   // channel factors kept in shared memory

__global__ void k_index(const double* __restrict__ uvw, const double* __restrict__ freq,
                        int64_t nrow, const int64_t* __restrict__ d_nrow, int nchan,
                        IndexParams p, gw_index_rec* __restrict__ out,
                        unsigned long long* __restrict__ dropped) {
    // [nc] channel factors f / c0, then [P - 1] plane thresholds as bit
    // patterns: non-negative finite doubles order like their int64 bits, so
    // the search compares integers (exactly the FP64 comparison)
    extern __shared__ double sh[];
    const int nc = min(nchan, kChanCache);
    const int nthr = p.P > 1 ? p.P - 1 : 0;
    double* sc = sh;
    long long* thr = reinterpret_cast<long long*>(sh + nc);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) sc[c] = __ddiv_rn(__ldg(freq + c), kC0);
    for (int j = threadIdx.x; j < nthr; j += blockDim.x) thr[j] = wplane_threshold(j, p);
    __syncthreads();
    if (d_nrow) nrow = min(nrow, *d_nrow);     // row count read on the device
    const int64_t nvis = nrow * (int64_t)nchan;
    unsigned int my_drops = 0;
    // (row, channel) of the grid-stride position, advanced without division
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t row = i / nchan;
    int chan = (int)(i - row * nchan);
    const int64_t srow = stride / nchan;
    const int schan = (int)(stride - srow * nchan);
    for (; i < nvis; i += stride) {
        const double f_c = chan < nc ? sc[chan] : __ddiv_rn(__ldg(freq + chan), kC0);
        gw_index_rec r;
        if (!index_record(__ldg(uvw + 3 * row + 0), __ldg(uvw + 3 * row + 1),
                          __ldg(uvw + 3 * row + 2), f_c, p, thr, r))
            ++my_drops;
        reinterpret_cast<int4*>(out)[i] = *reinterpret_cast<const int4*>(&r);
        row += srow;
        chan += schan;
        if (chan >= nchan) {
            chan -= nchan;
            ++row;
        }
    }
    // one atomic per warp
    for (int d = 16; d > 0; d >>= 1) my_drops += __shfl_down_sync(0xffffffffu, my_drops, d);
    if ((threadIdx.x & 31) == 0 && my_drops) atomicAdd(dropped, (unsigned long long)my_drops);
}

}  // namespace

void launch_index(const double* uvw, const double* freq, int64_t nrow, int nchan,
                  const IndexParams& prm, gw_index_rec* out, unsigned long long* dropped,
                  cudaStream_t s, const int64_t* d_nrow) {
    const int64_t nvis = nrow * (int64_t)nchan;
    if (nvis <= 0) return;
    const int threads = 256;
    int64_t blocks = (nvis + threads - 1) / threads;
    if (blocks > current_sm_count() * 16) blocks = current_sm_count() * 16;
    const size_t smem = sizeof(double) * (size_t)(std::min(nchan, kChanCache) +
                                                  (prm.P > 1 ? prm.P - 1 : 0));
    k_index<<<(unsigned)blocks, threads, smem, s>>>(uvw, freq, nrow, d_nrow, nchan, prm, out,
                                                    dropped);
    note_launch();
}

cudaError_t preload_index_kernels() {
    cudaFuncAttributes attr;
    return cudaFuncGetAttributes(&attr, k_index);
}

}  // namespace gw
