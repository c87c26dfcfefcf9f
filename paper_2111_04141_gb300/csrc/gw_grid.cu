// Gridding: table padding, visibility weighting and the dispatch to the
// gridding kernel instantiated per table kind (gw_grid_kernel.cuh).
#include "gw_internal.cuh"

namespace gw {

namespace {

// Zero-padded copy of the tables: slice (p, o) becomes (S + 6) rows x SP
// columns with the S x S values at row 3, column 7.
template <class T>
__global__ void k_pad_tables(const T* __restrict__ tab, const int64_t* __restrict__ plane_off,
                             const int64_t* __restrict__ pplane_off, const int* __restrict__ support,
                             int P, int beta, int SP, T* __restrict__ ptab) {
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
        T v{};
        if (row >= 0 && row < S && col >= 0 && col < S)
            v = tab[plane_off[p] + o * S * S + (int64_t)row * S + col];
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

}  // namespace

void launch_weight_vis(const void* vis, int kind, const float* w, int64_t n, float2* out,
                       cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > current_sm_count() * 16) blocks = current_sm_count() * 16;
    if (blocks < 1) blocks = 1;
    k_weight_vis<<<(unsigned)blocks, 256, 0, s>>>(vis, kind, w, n, out);
    note_launch();
}

int padded_stride(int smax) {
    const int need = smax + 14;
    for (int sp : {24, 32, 48, 80, 144}) if (need <= sp) return sp;
    return 272;
}

int64_t padded_table_elems(int S, int beta, int SP) { return (int64_t)beta * beta * (S + 6) * SP; }

void launch_pad_tables(const void* tab, int kind, const int64_t* plane_off,
                       const int64_t* pplane_off, const int* support, int P, int beta, int SP,
                       void* ptab, cudaStream_t s) {
    if (kind == GW_C64)
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
        default: launch_grid_c64(a, num_sms, s); break;
    }
}

}  // namespace gw
