// Internal declarations shared by the translation units of libgw.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstddef>

#include "gw.h"

namespace gw {

constexpr double kC0 = 299792458.0;   // speed of light, m/s
constexpr int kTile = 32;             // grid tile side of the degridding binner
constexpr int kGridTileU = 32;        // gridder tile: 32 (u) x 32 (v)
constexpr int kGridTileV = 32;
constexpr int kItemMax = 1024;        // max bin entries per gridder work item
constexpr double kQLimit = 1073741824.0;  // 2^30: |q| bound for a representable record

// Support of plane p: the odd integer nearest
// y = S_min + (S_max - S_min) p / (P - 1), ties upward: S = 2 floor(y/2) + 1,
// evaluated exactly in integers.
__host__ __device__ inline int plane_support(int p, int P, int smin, int smax) {
    if (P <= 1) return smin;
    long long Y = (long long)smin * (P - 1) + (long long)(smax - smin) * p;
    return (int)(2 * (Y / (2LL * (P - 1))) + 1);
}

__host__ __device__ inline long long floor_div(long long a, long long b) {
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

struct IndexParams {
    double L;        // field of view N * cell
    double halfN;    // N / 2 as double
    double beta_d;   // beta as double
    double Pm1_d;    // P - 1 as double
    double wmax;     // w_max (wavelengths)
    int N, beta, P, smin, smax;
};

// Work item of the gridder: a contiguous run of one tile's bin.
struct Item {
    int32_t tile;
    int32_t start;   // first entry index (absolute)
    int32_t len;     // number of entries (<= kItemMax)
    int32_t pad;
};

struct Scratch {
    gw_index_rec* rec = nullptr;      // [chunk] index records
    uint32_t* count = nullptr;        // [ntiles] bin sizes
    uint32_t* offsets = nullptr;      // [ntiles + 1] exclusive scan of count
    uint32_t* cursor = nullptr;       // [ntiles] scatter cursors
    uint32_t* item_off = nullptr;     // [ntiles + 1] exclusive scan of items per tile
    uint32_t* entries = nullptr;      // [entries_cap] binned visibility ids
    Item* items = nullptr;            // [items_cap]
    uint32_t* counters = nullptr;     // [4]: 0 = item queue head, 1..3 spare
    unsigned long long* dropped = nullptr;  // [1]
    unsigned long long* work = nullptr;     // [2]: valid visibilities, sum of S_p^2
    float2* wvis = nullptr;                 // [chunk * npol] weighted visibilities (lazy)
    int64_t entries_cap = 0;
    int64_t items_cap = 0;
};

// ---- launch counting -----------------------------------------------------
void note_launch(int n = 1);

// ---- index stage (gw_index.cu) --------------------------------------------
void launch_index(const double* uvw, const double* freq, int64_t nrow, int nchan,
                  const IndexParams& prm, gw_index_rec* out, unsigned long long* dropped,
                  cudaStream_t s);

// ---- binner (gw_bin.cu) ----------------------------------------------------
// mode 0: footprint tiles (every tile a record's footprint touches)
// mode 1: centre tile (the tile holding pixel (ku, kv))
// Tiles are 2^su (u) x 2^sv (v) pixels, ntu x ntv of them (row-major, v rows).
struct BinGeom {
    int mode, su, sv, ntu, ntv;
};
// Also accumulates sc.work[0] += valid records, sc.work[1] += sum of S_p^2.
// Work items are written only when sc.items is non-null.
void launch_bin(const gw_index_rec* rec, int64_t nvis, const BinGeom& g, int P, int smin, int smax,
                Scratch& sc, cudaStream_t s);

// ---- kernel tables (gw_tables.cu) -----------------------------------------
struct TableBuild {
    int N, beta, P, smin, smax;
    double field, wmax;
    const int* support;        // host [P]
    const double* wplane;      // host [P]
    const int64_t* plane_off;  // host [P + 1]
    int num_sms;
};
// Builds float2 tables (device, plane_off[P] complex elements) and the
// corrector h (device, N doubles and N floats).  Returns the global scale.
cudaError_t build_tables(const TableBuild& tb, float2* d_table, double* d_h, float* d_hf,
                         double* h_scale, cudaStream_t s);
int quad_nodes(double field, double w, int support, int smin);

// ---- gridding / degridding (gw_grid.cu, gw_degrid.cu) -----------------------
struct GridArgs {
    const gw_index_rec* rec;
    const float2* ptable;        // zero-padded tables (launch_pad_tables)
    const int64_t* pplane_off;   // device [P]: padded plane offsets
    const float2* vis;         // [nvis][npol]
    const float* weight;       // [nvis][npol] or null
    const float2* table;
    const int64_t* plane_off;  // device [P]
    const int* support;        // device [P]
    const uint32_t* entries;
    const Item* items;
    const uint32_t* item_count;  // device scalar: item_off[ntiles]
    uint32_t* queue;             // device scalar: work queue head (zeroed before launch)
    float2* grid;                // [npol][N][N]
    int N, npol, beta, ntiles_u;  // ntiles_u: gridder tiles along u
    int pad_stride;              // padded row stride (padded_stride(S_max))
};
void launch_grid(const GridArgs& a, int num_sms, cudaStream_t s);
// out[e] = vis[e] * w[e] (weights applied before gridding).
void launch_weight_vis(const float2* vis, const float* w, int64_t n, float2* out, cudaStream_t s);
// Zero-padded slice layout used by the gridder: (S + 6) rows x SP columns,
// SP = padded_stride(S_max) >= S_max + 14, one of a few compile-time strides.
int padded_stride(int smax);
int64_t padded_table_elems(int S, int beta, int SP);
void launch_pad_tables(const float2* tab, const int64_t* plane_off, const int64_t* pplane_off,
                       const int* support, int P, int beta, int SP, float2* ptab, cudaStream_t s);

struct DegridArgs {
    const gw_index_rec* rec;
    const float2* grid;
    const float2* table;
    const int64_t* plane_off;
    const int* support;
    const uint32_t* entries;    // centre-binned ids, offsets[ntiles] of them
    const uint32_t* n_entries;  // device scalar
    float2* vis_out;            // [nvis][npol]
    int N, npol, beta;
    // staged kernel only: work items over 16 x 16 centre tiles
    const Item* items = nullptr;
    const uint32_t* item_count = nullptr;
    uint32_t* queue = nullptr;
    int ntiles_u = 0;
};
void launch_degrid(const DegridArgs& a, int64_t nvis_upper, int num_sms, cudaStream_t s);
constexpr size_t kStagedSmemMax = 200 * 1024;   // staged-degrid region budget (bytes)
int degrid_staged_tile();
bool degrid_staged_fits(int hmax, int npol);
// Returns false (nothing launched) if the region does not fit.
bool launch_degrid_staged(const DegridArgs& a, int hmax, int num_sms, cudaStream_t s);

// ---- allocation-free scratch (gw_noalloc.cu) ------------------------------
// View of the file-scope static scratch on `device` (current); looks up the
// symbol's device address on first use per device.
cudaError_t static_scratch_view(int device, Scratch* sc);
int64_t static_scratch_max_vis();
int static_scratch_max_tiles();

// ---- correction (gw_correct.cu) -------------------------------------------
void launch_correct(float2* image, const float* h, int N, int npol, int mode, cudaStream_t s);
void launch_shift(float2* grid, int N, int npol, cudaStream_t s);

}  // namespace gw
