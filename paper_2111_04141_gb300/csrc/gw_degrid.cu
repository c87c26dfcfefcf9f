// Degridding kernel: the adjoint of gridding (operator G^T of Eq.
// (residualcalc), Section 1.6):
//     V[pol] = sum_{tv, tu} conj(K_i(tv, tu)) * G[pol][kv + tv][ku + tu],
// K_i the record's kernel (K_p[ov][ou], or its conjugate when w < 0).
//
// One warp per visibility: lanes stride over the taps of each footprint
// row, multiply-accumulate all polarisations, and reduce with warp
// shuffles.  Visibilities are visited in centre-tile order so that
// neighbouring warps read overlapping grid footprints from L1/L2.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kThreads = 256;

template <int NPOL>
__global__ void __launch_bounds__(kThreads) k_degrid(DegridArgs a) {
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
        const float2* K = a.table + __ldg(a.plane_off + r.plane) +
                          ((int64_t)(r.ov + hb) * a.beta + (r.ou + hb)) * S * S;
        // conj(K_i): K_i = K for w >= 0 (use conj K), K_i = conj K for w < 0 (use K)
        const float s = (r.flags & GW_FLAG_CONJ) ? -1.f : 1.f;
        float acc[NPOL][2];
#pragma unroll
        for (int p = 0; p < NPOL; ++p) acc[p][0] = acc[p][1] = 0.f;
        for (int tv = 0; tv < S; ++tv) {
            const int64_t row = r.kv - h + tv;
            for (int tu = lane; tu < S; tu += 32) {
                const float2 k = __ldg(K + tv * S + tu);
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
            a.vis_out[(int64_t)id * NPOL + lane] = make_float2(re, im);
        }
    }
}

template <int NPOL>
void launch_t(const DegridArgs& a, int64_t nvis, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid<NPOL>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (nvis * 32 + kThreads - 1) / kThreads;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms * per_sm);
    if (blocks < 1) blocks = 1;
    k_degrid<NPOL><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    note_launch();
}

}  // namespace

void launch_degrid(const DegridArgs& a, int64_t nvis, int num_sms, cudaStream_t s) {
    switch (a.npol) {
        case 1: launch_t<1>(a, nvis, num_sms, s); break;
        case 2: launch_t<2>(a, nvis, num_sms, s); break;
        case 3: launch_t<3>(a, nvis, num_sms, s); break;
        default: launch_t<4>(a, nvis, num_sms, s); break;
    }
}

}  // namespace gw
