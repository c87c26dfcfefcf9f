// Gridding: table padding, visibility weighting and the dispatch to the
// gridding kernel instantiated per table kind (gw_grid_kernel.cuh).
#include "gw_internal.cuh"

namespace gw {

namespace {

// Zero-padded copy of the tables: slice (p, o) becomes (S + 2 kGridPadR)
// rows x SP columns with the S x S values at row kGridPadR, column kGridPadC
// (3 and 7 for the 8 x 4 lane layout).
template <class T>
__global__ void k_pad_tables(const T* __restrict__ tab, const int64_t* __restrict__ plane_off,
                             const int64_t* __restrict__ pplane_off, const int* __restrict__ support,
                             int P, int beta, int SP, T* __restrict__ ptab) {
    const int p = blockIdx.y;
    if (p >= P) return;
    const int S = support[p], SR = S + 2 * kGridPadR;
    const int64_t per = (int64_t)SR * SP;
    const int64_t n = (int64_t)beta * beta * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = e / per;
        const int rem = (int)(e - o * per);
        const int row = rem / SP - kGridPadR, col = rem % SP - kGridPadC;
        T v{};
        if (row >= 0 && row < S && col >= 0 && col < S)
            v = tab[plane_off[p] + o * S * S + (int64_t)row * S + col];
        ptab[pplane_off[p] + e] = v;
    }
}

// The same padding for a real kernel: the real parts of an FP32 table.
__global__ void k_pad_tables_real(const float2* __restrict__ tab, const int64_t* __restrict__ plane_off,
                                  const int64_t* __restrict__ pplane_off,
                                  const int* __restrict__ support, int P, int beta, int SP,
                                  float* __restrict__ ptab) {
    const int p = blockIdx.y;
    if (p >= P) return;
    const int S = support[p], SR = S + 2 * kGridPadR;
    const int64_t per = (int64_t)SR * SP;
    const int64_t n = (int64_t)beta * beta * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = e / per;
        const int rem = (int)(e - o * per);
        const int row = rem / SP - kGridPadR, col = rem % SP - kGridPadC;
        float v = 0.f;
        if (row >= 0 && row < S && col >= 0 && col < S)
            v = tab[plane_off[p] + o * S * S + (int64_t)row * S + col].x;
        ptab[pplane_off[p] + e] = v;
    }
}

__global__ void k_weight_vis(const void* __restrict__ vis, int kind, const float* __restrict__ w,
                             int64_t n, float2* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = load_vis(vis, kind, e);
        const float s = w[e];
        out[e] = make_float2(v.x * s, v.y * s);
    }
}

// Direct gridding for small inputs: no binning, one warp per visibility,
// whose lane 0 computes the visibility's index record (the same bit-exact
// FP64 sequence as the index stage) and broadcasts it, then spreads it over
// the flattened S x S taps of its (unpadded) kernel slice with one global
// vector atomic per tap and polarisation.  One launch per call instead of
// the binned path's seven, which is what small jobs pay for.  Counts the
// dropped visibilities and accumulates the work counters the binner would
// (valid records, sum of S^2).
constexpr int kDirectChanCache = 256;   // channel factors kept in shared memory

template <int NPOL, int TK>
__global__ void __launch_bounds__(256) k_grid_direct(GridArgs a, const void* __restrict__ table,
                                                     DirectIndex di,
                                                     unsigned long long* __restrict__ work) {
    using TE = TabElem<TK>;
    // [P - 1] w-plane thresholds as int64 bit patterns and [nc] channel
    // factors f / c0, as the index stage builds them
    extern __shared__ long long sh_idx[];
    __shared__ unsigned long long s_cnt[3];   // the block's valid, taps, dropped
    const int nthr = di.p.P > 1 ? di.p.P - 1 : 0;
    const int nc = min(di.nchan, kDirectChanCache);
    long long* thr = sh_idx;
    double* fc = reinterpret_cast<double*>(sh_idx + nthr);
    for (int j = threadIdx.x; j < nthr; j += blockDim.x) thr[j] = wplane_threshold(j, di.p);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) fc[c] = __ddiv_rn(__ldg(di.freq + c), kC0);
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int hb = a.beta / 2, N = a.N;
    const int64_t nvis = di.nrow * (int64_t)di.nchan;
    unsigned long long n_valid = 0, n_taps = 0, n_drop = 0;
    for (int64_t i = warp0; i < nvis; i += nwarps) {
        int4 rv = make_int4(0, 0, 0, 0);
        if (lane == 0) {
            const int64_t row = i / di.nchan;
            const int chan = (int)(i - row * di.nchan);
            const double f_c = chan < nc ? fc[chan] : __ddiv_rn(__ldg(di.freq + chan), kC0);
            gw_index_rec r;
            index_record(__ldg(di.uvw + 3 * row + 0), __ldg(di.uvw + 3 * row + 1),
                         __ldg(di.uvw + 3 * row + 2), f_c, di.p, thr, r);
            rv = *reinterpret_cast<const int4*>(&r);
        }
        rv.x = __shfl_sync(0xffffffffu, rv.x, 0);
        rv.y = __shfl_sync(0xffffffffu, rv.y, 0);
        rv.z = __shfl_sync(0xffffffffu, rv.z, 0);
        rv.w = __shfl_sync(0xffffffffu, rv.w, 0);
        const gw_index_rec rc = *reinterpret_cast<const gw_index_rec*>(&rv);
        if (!(rc.flags & GW_FLAG_VALID)) {
            if (lane == 0) ++n_drop;
            continue;
        }
        const int plane = a.layer_tiles ? 0 : rc.plane;
        const int S = __ldg(a.support + plane), h = S >> 1;
        if (lane == 0) {
            ++n_valid;
            n_taps += (unsigned long long)(S * S);
        }
        const int64_t kofs = __ldg(a.plane_off + plane) +
                             ((int64_t)(rc.ov + hb) * a.beta + (rc.ou + hb)) * S * S;
#ifdef GW_DEBUG_BOUNDS
        // the slice and the footprint's pixels
        if (!gw_in_bounds((a.table_elems == 0 || (kofs >= 0 && kofs + (int64_t)S * S <= a.table_elems)) &&
                              rc.ku - h >= 0 && rc.ku + h < N && rc.kv - h >= 0 && rc.kv + h < N,
                          a.queue ? a.queue + 1 : nullptr))
            continue;
#endif
        const typename TE::T* K = reinterpret_cast<const typename TE::T*>(table) + kofs;
        const float sg = (rc.flags & GW_FLAG_CONJ) ? -1.f : 1.f;
        float2 V[NPOL];
#pragma unroll
        for (int p = 0; p < NPOL; ++p) {
            V[p] = load_vis(a.vis, a.vis_kind, i * NPOL + p);
            if (a.weight) {
                const float w = __ldg(a.weight + i * NPOL + p);
                V[p].x *= w;
                V[p].y *= w;
            }
        }
        float2* const gbase = a.grid + (a.layer_tiles ? (int64_t)rc.plane * a.layer_stride : 0);
        for (int t = lane; t < S * S; t += 32) {
            const int tv = t / S, tu = t - tv * S;
            const float2 k = TE::load(K + t);
            const float kr = k.x * a.table_inv, ki = sg * k.y * a.table_inv;
            const int64_t pix = (int64_t)(rc.kv - h + tv) * N + (rc.ku - h + tu);
#pragma unroll
            for (int p = 0; p < NPOL; ++p) {
                const float2 val = make_float2(kr * V[p].x - ki * V[p].y, kr * V[p].y + ki * V[p].x);
                const int64_t off = (int64_t)p * N * N + pix;
                if (a.grid_err) {
                    const float2 old = atomicAdd(gbase + off, val);
                    // compensated commit, as in the binned kernel
                    float2 e;
                    {
                        const float s_ = __fadd_rn(old.x, val.x);
                        const float bv = __fsub_rn(s_, old.x);
                        const float av = __fsub_rn(s_, bv);
                        e.x = __fadd_rn(__fsub_rn(old.x, av), __fsub_rn(val.x, bv));
                    }
                    {
                        const float s_ = __fadd_rn(old.y, val.y);
                        const float bv = __fsub_rn(s_, old.y);
                        const float av = __fsub_rn(s_, bv);
                        e.y = __fadd_rn(__fsub_rn(old.y, av), __fsub_rn(val.y, bv));
                    }
                    if (e.x != 0.f || e.y != 0.f) atomicAdd(a.grid_err + off, e);
                } else {
                    atomicAdd(gbase + off, val);
                }
            }
        }
    }
    // counts are held by lane 0 of each warp: summed per block first, so
    // the global counters take one atomic per block
    if (lane == 0) {
        if (n_valid) {
            atomicAdd(&s_cnt[0], n_valid);
            atomicAdd(&s_cnt[1], n_taps);
        }
        if (n_drop) atomicAdd(&s_cnt[2], n_drop);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cnt[0]) {
            atomicAdd(work, s_cnt[0]);
            atomicAdd(work + 1, s_cnt[1]);
        }
        if (s_cnt[2]) atomicAdd(di.dropped, s_cnt[2]);
    }
}

template <int TK>
void launch_direct_k(const GridArgs& a, const void* table, const DirectIndex& di,
                     unsigned long long* work, cudaStream_t s) {
    const int64_t nvis = di.nrow * (int64_t)di.nchan;
    int64_t blocks = (nvis * 32 + 255) / 256;
    if (blocks > current_sm_count() * 8) blocks = current_sm_count() * 8;
    if (blocks < 1) blocks = 1;
    const size_t smem = sizeof(long long) * (size_t)(di.p.P > 1 ? di.p.P - 1 : 0) +
                        sizeof(double) * (size_t)std::min(di.nchan, kDirectChanCache);
    switch (a.npol) {
        case 1: k_grid_direct<1, TK><<<(unsigned)blocks, 256, smem, s>>>(a, table, di, work); break;
        case 2: k_grid_direct<2, TK><<<(unsigned)blocks, 256, smem, s>>>(a, table, di, work); break;
        case 3: k_grid_direct<3, TK><<<(unsigned)blocks, 256, smem, s>>>(a, table, di, work); break;
        default: k_grid_direct<4, TK><<<(unsigned)blocks, 256, smem, s>>>(a, table, di, work); break;
    }
    note_launch();
}

}  // namespace

void launch_grid_direct(const GridArgs& a, const void* table, const DirectIndex& di,
                        unsigned long long* work, cudaStream_t s) {
    if (di.nrow <= 0 || di.nchan <= 0) return;
    switch (a.table_kind) {
        case GW_BF16X2: launch_direct_k<GW_BF16X2>(a, table, di, work, s); break;
        case GW_F16X2: launch_direct_k<GW_F16X2>(a, table, di, work, s); break;
        default: launch_direct_k<GW_C64>(a, table, di, work, s); break;
    }
}

void launch_weight_vis(const void* vis, int kind, const float* w, int64_t n, float2* out,
                       cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > current_sm_count() * 16) blocks = current_sm_count() * 16;
    if (blocks < 1) blocks = 1;
    k_weight_vis<<<(unsigned)blocks, 256, 0, s>>>(vis, kind, w, n, out);
    note_launch();
}

int padded_stride(int smax) {
    const int need = smax + 2 * kGridPadC;
#if GW_GRID_LANES_U == 16
    for (int sp : {32, 48, 64, 96, 160}) if (need <= sp) return sp;
    return 288;
#else
    for (int sp : {24, 32, 48, 80, 144}) if (need <= sp) return sp;
    return 272;
#endif
}

int64_t padded_table_elems(int S, int beta, int SP) {
    return (int64_t)beta * beta * (S + 2 * kGridPadR) * SP;
}

void launch_pad_tables(const void* tab, int kind, const int64_t* plane_off,
                       const int64_t* pplane_off, const int* support, int P, int beta, int SP,
                       void* ptab, cudaStream_t s) {
    if (kind == kTabRealF32)
        k_pad_tables_real<<<dim3(256, P), 256, 0, s>>>(
            static_cast<const float2*>(tab), plane_off, pplane_off, support, P, beta, SP,
            static_cast<float*>(ptab));
    else if (kind == GW_C64)
        k_pad_tables<float2><<<dim3(256, P), 256, 0, s>>>(
            static_cast<const float2*>(tab), plane_off, pplane_off, support, P, beta, SP,
            static_cast<float2*>(ptab));
    else
        k_pad_tables<uint32_t><<<dim3(256, P), 256, 0, s>>>(
            static_cast<const uint32_t*>(tab), plane_off, pplane_off, support, P, beta, SP,
            static_cast<uint32_t*>(ptab));
    note_launch();
}

void launch_grid(const GridArgs& a, int num_sms, cudaStream_t s) {
    cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
    switch (a.table_kind) {
        case GW_BF16X2: launch_grid_bf16(a, num_sms, s); break;
        case GW_F16X2: launch_grid_f16(a, num_sms, s); break;
        case kTabRealF32: launch_grid_r32(a, num_sms, s); break;
        default: launch_grid_c64(a, num_sms, s); break;
    }
}

}  // namespace gw
