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

struct AxisIdx {
    long long k, o;
    bool ok;
};

constexpr int kChanCache = 1024;   // channel factors kept in shared memory

__device__ __forceinline__ AxisIdx axis_index(double coord_m, double sc, const IndexParams& p) {
    // u_lambda = u * (f / c0) ; x = u_lambda * L + N/2 ; q = floor(beta * x + 0.5)
    const double lam = __dmul_rn(coord_m, sc);
    const double x = __dadd_rn(__dmul_rn(lam, p.L), p.halfN);
    const double q = floor(__dadd_rn(__dmul_rn(p.beta_d, x), 0.5));
    AxisIdx r;
    r.ok = isfinite(q) && fabs(q) < kQLimit;
    const long long qi = r.ok ? (long long)q : 0LL;
    r.k = floor_div(qi + p.beta / 2, p.beta);
    r.o = qi - r.k * p.beta;
    return r;
}

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
    for (int j = threadIdx.x; j < nthr; j += blockDim.x) {
        const double t = __ddiv_rn((double)j + 0.5, p.Pm1_d);      // (j + 1) - 1/2, exact
        thr[j] = __double_as_longlong(__dmul_rn(__dmul_rn(t, t), p.wmax));
    }
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
        const double u = __ldg(uvw + 3 * row + 0);
        const double v = __ldg(uvw + 3 * row + 1);
        const AxisIdx au = axis_index(u, f_c, p);
        const AxisIdx av = axis_index(v, f_c, p);
        int plane = 0;
        bool conj = false, okw = true;
        if (p.P > 1) {
            const double wl = __dmul_rn(__ldg(uvw + 3 * row + 2), f_c);
            okw = isfinite(wl);
            if (okw) {
                // number of thresholds <= |w| (first index with thr > |w|)
                const long long a = __double_as_longlong(fabs(wl));
                int lo = 0, hi = nthr;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (thr[mid] <= a) lo = mid + 1; else hi = mid;
                }
                plane = lo;
            }
            conj = wl < 0.0;
        } else if (p.nlayers > 0) {
            // w-stacking layer: nearest of w_l = wmin + l dw, clamped to the layers
            const double wl = __dmul_rn(__ldg(uvw + 3 * row + 2), f_c);
            const double t = floor(__dadd_rn(__ddiv_rn(__dsub_rn(wl, p.wmin), p.dw), 0.5));
            okw = isfinite(t);
            plane = okw ? (int)fmin(fmax(t, 0.0), (double)(p.nlayers - 1)) : 0;
        }
        const int h = plane_support(plane, p.P, p.smin, p.smax) / 2;
        const bool inside = (au.k - h >= 0) && (au.k + h <= p.N - 1) &&
                            (av.k - h >= 0) && (av.k + h <= p.N - 1);
        const bool valid = au.ok && av.ok && okw && inside;
        gw_index_rec r;
        if (valid) {
            r.ku = (int32_t)au.k;
            r.kv = (int32_t)av.k;
            r.ou = (int16_t)au.o;
            r.ov = (int16_t)av.o;
            r.plane = (int16_t)plane;
            r.flags = (uint16_t)(GW_FLAG_VALID | (conj ? GW_FLAG_CONJ : 0u));
        } else {
            r.ku = r.kv = 0;
            r.ou = r.ov = 0;
            r.plane = 0;
            r.flags = 0;
            ++my_drops;
        }
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
