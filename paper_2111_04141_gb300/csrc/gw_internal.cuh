// Internal declarations shared by the translation units of libgw.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstddef>

#include "gw.h"

namespace gw {

constexpr double kC0 = 299792458.0;   // speed of light, m/s
constexpr int kTile = 32;             // grid tile side of the degridding binner
#ifndef GW_GRID_TILE_SHIFT_U
#define GW_GRID_TILE_SHIFT_U 6
#endif
constexpr int kGridTileShiftU = GW_GRID_TILE_SHIFT_U;
constexpr int kGridTileU = 1 << kGridTileShiftU;   // gridder tile: kGridTileU (u) x 32 (v)
constexpr int kGridTileV = 32;
// Gridder lane layout: a compute warp's 32 lanes are kGridLanesU (u) x
// kGridLanesV (v) grid points, and each lane holds 4 of them kGridLanesV
// rows apart, so a warp owns a kGridLanesU x 4 kGridLanesV block.  The padded
// tables carry kGridLanesV - 1 zero rows above and below each slice and at
// least kGridLanesU - 1 zero columns on each side (the lanes of a loaded slot
// reach that far past the footprint).
#ifndef GW_GRID_LANES_U
#define GW_GRID_LANES_U 8
#endif
constexpr int kGridLanesU = GW_GRID_LANES_U;
constexpr int kGridLanesV = 32 / kGridLanesU;
constexpr int kGridPadR = kGridLanesV - 1;
constexpr int kGridPadC = kGridLanesU - 1;
constexpr int kItemMax = 1024;        // default max bin entries per work item
constexpr int kItemMin = 64;          // smallest work-item size a plan may be tuned to
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

// ---- storage types ---------------------------------------------------------
// Tables and visibilities are stored as complex FP32 (float2) or as pairs of
// 16-bit floats (re in the low half of a 32-bit word, im in the high half);
// arithmetic is always FP32.
__host__ __device__ constexpr int dtype_bytes(int kind) { return kind == GW_C64 ? 8 : 4; }

__device__ __forceinline__ float2 unpack_bf16x2(uint32_t u) {
    // a bfloat16 is the upper half of the float32 with the same bits
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
__device__ __forceinline__ float2 unpack_f16x2(uint32_t u) {
    __half2 h;
    memcpy(&h, &u, sizeof u);
    return __half22float2(h);
}

// Gridder table kind of the real w = 0 kernel (2-D plans with FP32 tables):
// the padded gridder table holds the real parts only, the imaginary parts of
// that kernel being exactly zero (no w-screen phase, cosine transform).
constexpr int kTabRealF32 = 3;

// Table element of kind TK and its load (read-only path); kReal: the
// imaginary part is zero and its FMAs are left out.
template <int TK> struct TabElem;
template <> struct TabElem<GW_C64> {
    static constexpr bool kReal = false;
    using T = float2;
    static __device__ __forceinline__ float2 cvt(T v) { return v; }
    static __device__ __forceinline__ float2 load(const T* p) { return __ldg(p); }
};
template <> struct TabElem<GW_BF16X2> {
    static constexpr bool kReal = false;
    using T = uint32_t;
    static __device__ __forceinline__ float2 cvt(T v) { return unpack_bf16x2(v); }
    static __device__ __forceinline__ float2 load(const T* p) { return unpack_bf16x2(__ldg(p)); }
};
template <> struct TabElem<GW_F16X2> {
    static constexpr bool kReal = false;
    using T = uint32_t;
    static __device__ __forceinline__ float2 cvt(T v) { return unpack_f16x2(v); }
    static __device__ __forceinline__ float2 load(const T* p) { return unpack_f16x2(__ldg(p)); }
};
template <> struct TabElem<kTabRealF32> {
    static constexpr bool kReal = true;
    using T = float;
    static __device__ __forceinline__ float2 cvt(T v) { return make_float2(v, 0.f); }
    static __device__ __forceinline__ float2 load(const T* p) { return make_float2(__ldg(p), 0.f); }
};

// Visibility i of a buffer of kind `kind` (uniform runtime branch).
__device__ __forceinline__ float2 load_vis(const void* vis, int kind, int64_t i) {
    if (kind == GW_C64) return __ldg(reinterpret_cast<const float2*>(vis) + i);
    const uint32_t u = __ldg(reinterpret_cast<const uint32_t*>(vis) + i);
    return kind == GW_BF16X2 ? unpack_bf16x2(u) : unpack_f16x2(u);
}

// Store (re, im) as element i of a buffer of kind `kind`, rounded to nearest.
__device__ __forceinline__ void store_vis(void* vis, int kind, int64_t i, float re, float im) {
    if (kind == GW_C64) {
        reinterpret_cast<float2*>(vis)[i] = make_float2(re, im);
    } else if (kind == GW_BF16X2) {
        reinterpret_cast<__nv_bfloat162*>(vis)[i] = __floats2bfloat162_rn(re, im);
    } else {
        reinterpret_cast<__half2*>(vis)[i] = __floats2half2_rn(re, im);
    }
}

struct IndexParams {
    double L;        // field of view N * cell
    double halfN;    // N / 2 as double
    double beta_d;   // beta as double
    double Pm1_d;    // P - 1 as double
    double wmax;     // w_max (wavelengths)
    int N, beta, P, smin, smax;
    // w-stacking (2-D plans only): layer = clamp(floor((w - wmin) / dw + 1/2), 0, nlayers - 1)
    // stored in the record's `plane` field; nlayers = 0: off
    int nlayers = 0;
    double wmin = 0.0, dw = 1.0;
};

// The index record of one visibility (Section 3.3.5 pre-processing, Section
// 2.3.6 NN lookup, Section 2.3.1 bounded records): every floating-point step
// an explicitly rounded FP64 intrinsic, so the result is bit-exact with any
// IEEE-754 implementation of the same sequence.  f_c = f / c0 of the
// visibility's channel; thr[0 .. P - 2] are the w-plane thresholds
// ((j + 1/2) / (P - 1))^2 w_max as int64 bit patterns (non-negative finite
// doubles order like their bits).  Returns false (and an all-zero record)
// for a dropped visibility.
struct IndexAxis {
    long long k, o;
    bool ok;
};
__device__ __forceinline__ IndexAxis index_axis(double coord_m, double f_c, const IndexParams& p) {
    // u_lambda = u * (f / c0) ; x = u_lambda * L + N/2 ; q = floor(beta * x + 0.5)
    const double lam = __dmul_rn(coord_m, f_c);
    const double x = __dadd_rn(__dmul_rn(lam, p.L), p.halfN);
    const double q = floor(__dadd_rn(__dmul_rn(p.beta_d, x), 0.5));
    IndexAxis r;
    r.ok = isfinite(q) && fabs(q) < kQLimit;
    const long long qi = r.ok ? (long long)q : 0LL;
    r.k = floor_div(qi + p.beta / 2, p.beta);
    r.o = qi - r.k * p.beta;
    return r;
}
__device__ __forceinline__ bool index_record(double u, double v, double w, double f_c,
                                             const IndexParams& p, const long long* thr,
                                             gw_index_rec& r) {
    const IndexAxis au = index_axis(u, f_c, p);
    const IndexAxis av = index_axis(v, f_c, p);
    int plane = 0;
    bool conj = false, okw = true;
    if (p.P > 1) {
        const double wl = __dmul_rn(w, f_c);
        okw = isfinite(wl);
        if (okw) {
            // number of thresholds <= |w| (first index with thr > |w|)
            const long long a = __double_as_longlong(fabs(wl));
            int lo = 0, hi = p.P - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (thr[mid] <= a) lo = mid + 1; else hi = mid;
            }
            plane = lo;
        }
        conj = wl < 0.0;
    } else if (p.nlayers > 0) {
        // w-stacking layer: nearest of w_l = wmin + l dw, clamped to the layers
        const double wl = __dmul_rn(w, f_c);
        const double t = floor(__dadd_rn(__ddiv_rn(__dsub_rn(wl, p.wmin), p.dw), 0.5));
        okw = isfinite(t);
        plane = okw ? (int)fmin(fmax(t, 0.0), (double)(p.nlayers - 1)) : 0;
    }
    const int h = plane_support(plane, p.P, p.smin, p.smax) / 2;
    const bool inside = (au.k - h >= 0) && (au.k + h <= p.N - 1) &&
                        (av.k - h >= 0) && (av.k + h <= p.N - 1);
    const bool valid = au.ok && av.ok && okw && inside;
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
    }
    return valid;
}
// Threshold j of the w-plane search (as its int64 bit pattern).
__device__ __forceinline__ long long wplane_threshold(int j, const IndexParams& p) {
    const double t = __ddiv_rn((double)j + 0.5, p.Pm1_d);      // (j + 1) - 1/2, exact
    return __double_as_longlong(__dmul_rn(__dmul_rn(t, t), p.wmax));
}

// Work item of the gridder: a contiguous run of one tile's bin.
struct Item {
    int32_t tile;
    int32_t start;   // first entry index (absolute)
    int32_t len;     // number of entries (<= the geometry's item_max)
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
    uint32_t* scan_tmp = nullptr;           // [scan_tmp_words(scan_tmp_bins)] segment totals,
                                            // or null (single-CTA scan)
    int64_t scan_tmp_bins = 0;              // bins scan_tmp is sized for
    int64_t entries_cap = 0;
    int64_t items_cap = 0;
};

// ---- launch counting -----------------------------------------------------
void note_launch(int n = 1);

// SM count of the current device (cached per device); grid-stride kernels
// size their grids as a multiple of it.
int current_sm_count();

// ---- allocations -----------------------------------------------------------
// Every device allocation of the library goes through dev_alloc and every
// host allocation of a plan object checks alloc_fault(), so a test can make
// the n-th allocation from now fail on the host (gw_debug_fail_alloc)
// without touching the GPU.
bool alloc_fault();
cudaError_t dev_alloc(void** ptr, size_t bytes);
void dev_free(void* ptr);   // frees a dev_alloc allocation (null accepted)

// Row count read on the device when kernels run (graph replays with any
// count up to the captured maximum); nrow == null: the host count is used.
struct DevCount {
    const int64_t* nrow = nullptr;
    int nchan = 1;
    __device__ __forceinline__ int64_t clamp(int64_t nvis_max) const {
        if (!nrow) return nvis_max;
        const int64_t n = *nrow * (int64_t)nchan;
        return n < nvis_max ? (n > 0 ? n : 0) : nvis_max;
    }
};

// ---- index stage (gw_index.cu) --------------------------------------------
void launch_index(const double* uvw, const double* freq, int64_t nrow, int nchan,
                  const IndexParams& prm, gw_index_rec* out, unsigned long long* dropped,
                  cudaStream_t s, const int64_t* d_nrow = nullptr);

// ---- binner (gw_bin.cu) ----------------------------------------------------
// mode 0: footprint tiles (every tile a record's footprint touches)
// mode 1: centre tile (the tile holding pixel (ku, kv))
// Tiles are 2^su (u) x 2^sv (v) pixels, ntu x ntv of them (row-major, v rows);
// each tile's bin is cut into work items of at most item_max entries.
struct BinGeom {
    int mode, su, sv, ntu, ntv;
    int item_max = kItemMax;
    int layer_tiles = 0;   // > 0: tile id += (record.plane / group_planes) * layer_tiles
    int nlayers = 1;       // layers binned when layer_tiles > 0 (ntu * ntv * nlayers tiles)
    int group_planes = 1;  // planes per layer: 1 for w-stacking layers, more for plane groups
};
// Words of Scratch::scan_tmp for a multi-CTA scan over ntiles bins.
int64_t scan_tmp_words(int64_t ntiles);
// Also accumulates sc.work[0] += valid records, sc.work[1] += sum of S_p^2.
// Work items are written only when sc.items is non-null.
void launch_bin(const gw_index_rec* rec, int64_t nvis, const BinGeom& g, int P, int smin, int smax,
                Scratch& sc, cudaStream_t s, DevCount dc = DevCount{});

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
// With d_table16 non-null it also stores every entry, scaled by 2^exp2, as a
// 16-bit pair of kind kind16 (GW_BF16X2 or GW_F16X2), rounded once from FP64;
// exp2 is 0 for bfloat16 and, for float16, puts the largest entry (the
// w = 0, o = 0 centre tap) in [2^14, 2^15) so no entry overflows and small
// ones stay clear of the subnormal range.
cudaError_t build_tables(const TableBuild& tb, float2* d_table, uint32_t* d_table16, int kind16,
                         double* d_h, float* d_hf, double* h_scale, int* h_exp2, double* d_c1,
                         cudaStream_t s);
// d_c1 (optional, beta * support[0] doubles): the unnormalised 1-D w = 0
// kernel C(f / beta) at fine offsets f = fmin .. fmin + F - 1, fmin = -beta h - beta/2 + 1.
// Hybrid pruner (Section 2.4): Z table [beta/2][sz] (float) and the pruning
// corrector h_pr [N] (FP64 and FP32).  Synchronous.
cudaError_t build_prune(int sz, int beta, int N, float* d_z, double* d_hpr, float* d_hprf,
                        cudaStream_t s);
int quad_nodes(double field, double w, int support, int smin);

// ---- gridding / degridding (gw_grid.cu, gw_degrid.cu) -----------------------
struct GridArgs {
    const gw_index_rec* rec;
    const void* ptable;          // zero-padded tables of kind table_kind (launch_pad_tables)
    const int64_t* pplane_off;   // device [P]: padded plane offsets
    const void* vis;           // [nvis][npol] of kind vis_kind
    const float* weight;       // [nvis][npol] or null
    const int64_t* plane_off;  // device [P]
    const int* support;        // device [P]
    const uint32_t* entries;
    const Item* items;
    const uint32_t* item_count;  // device scalar: item_off[ntiles] (one past the last item)
    const uint32_t* item_first = nullptr;  // device scalar: first item (null: 0)
    int64_t ptable_elems = 0;    // elements of ptable (debug bounds checks)
    int64_t table_elems = 0;     // elements of the unpadded table (direct path; checks)
    uint32_t* queue;             // device words: [0] work queue head (zeroed before launch),
                                 // [1] status (bit 0 set when a bounded device wait gave up)
    float2* grid;                // [npol][N][N]
    float2* grid_err;            // [npol][N][N] commit rounding errors, or null (plain commits)
    int N, npol, beta, ntiles_u;  // ntiles_u: gridder tiles along u
    int pad_stride;              // padded row stride (padded_stride(S_max))
    int vis_kind, table_kind;    // gw_dtype of vis and of the tables
    float table_inv;             // 2^-exp2: undoes the table storage scale at the commit
    // w-stacking: tile ids are layer * layer_tiles + tile, records carry their
    // layer in `plane`, layer grids are layer_stride elements apart (0 = off)
    int layer_tiles = 0;
    int64_t layer_stride = 0;
    // plane groups: tile ids are group * layer_tiles + tile as above, but the
    // records keep their own w-plane and every group adds into `grid`
    // (layer_stride 0)
    int plane_groups = 0;
};
void launch_grid(const GridArgs& a, int num_sms, cudaStream_t s);
// Direct gridding (no bins) of nrow x nchan visibilities, each warp
// computing its visibility's index record: `table` is the unpadded table of
// kind a.table_kind; adds the dropped visibilities to *dropped, and to
// work[0] (valid records) and work[1] (sum of S_p^2).  For inputs small
// enough that launches dominate.
struct DirectIndex {
    const double* uvw;       // [nrow][3] metres (device)
    const double* freq;      // [nchan] Hz (device)
    int64_t nrow;
    int nchan;
    IndexParams p;
    unsigned long long* dropped;
};
void launch_grid_direct(const GridArgs& a, const void* table, const DirectIndex& di,
                        unsigned long long* work, cudaStream_t s);
// Direct gridding is chosen for at most this many visibilities per chunk and
// this many tap updates (visibilities x S_max^2 x npol).
constexpr int64_t kDirectMaxVis = 16384;
// Plane groups of the binned gridder: at most this many, chosen
// automatically when FP32 padded tables exceed kGroupTableBytes (about the
// L2), with about kGroupTargetBytes of tables per group.
constexpr int kMaxPlaneGroups = 16;
constexpr int64_t kGroupTableBytes = 128ll << 20;
constexpr int64_t kGroupTargetBytes = 64ll << 20;
// Bands of tile rows a banded read-back may use (gw_grid_vis_devcount_readback).
constexpr int kReadbackBandsMax = 64;
constexpr int64_t kDirectMaxTaps = (int64_t)1 << 22;
// One instantiation set per table kind (gw_grid_c64.cu, gw_grid_bf16.cu, gw_grid_f16.cu,
// gw_grid_r32.cu).
void launch_grid_c64(const GridArgs& a, int num_sms, cudaStream_t s);
void launch_grid_r32(const GridArgs& a, int num_sms, cudaStream_t s);
void launch_grid_bf16(const GridArgs& a, int num_sms, cudaStream_t s);
void launch_grid_f16(const GridArgs& a, int num_sms, cudaStream_t s);
// out[e] = vis[e] * w[e] in FP32 (weights applied before gridding); vis of kind `kind`.
void launch_weight_vis(const void* vis, int kind, const float* w, int64_t n, float2* out,
                       cudaStream_t s);
// Zero-padded slice layout used by the gridder: (S + 6) rows x SP columns,
// SP = padded_stride(S_max) >= S_max + 14, one of a few compile-time strides.
int padded_stride(int smax);
int64_t padded_table_elems(int S, int beta, int SP);
// tab/ptab hold elements of kind `kind` (8 bytes for GW_C64, else 4).
void launch_pad_tables(const void* tab, int kind, const int64_t* plane_off,
                       const int64_t* pplane_off, const int* support, int P, int beta, int SP,
                       void* ptab, cudaStream_t s);

struct DegridArgs {
    const gw_index_rec* rec;
    const float2* grid;
    const void* table;          // unpadded tables of kind table_kind
    const int64_t* plane_off;
    const int* support;
    const uint32_t* entries;    // centre-binned ids, offsets[ntiles] of them
    const uint32_t* n_entries;  // device scalar
    void* vis_out;              // [nvis][npol] of kind vis_kind
    int N, npol, beta;
    int vis_kind = GW_C64, table_kind = GW_C64;
    float table_inv = 1.f;      // 2^-exp2: undoes the table storage scale
    // staged kernel only: work items over 16 x 16 centre tiles
    const Item* items = nullptr;
    const uint32_t* item_count = nullptr;
    uint32_t* queue = nullptr;
    int ntiles_u = 0;
    // debug bounds checks (0: unknown, not checked)
    int64_t table_elems = 0;    // elements of `table`, slack included
    int64_t vis_count = 0;      // visibilities of vis_out
};
void launch_degrid(const DegridArgs& a, int64_t nvis_upper, int num_sms, cudaStream_t s);
// Staged-degrid region budget (bytes): the 227 KB a CTA may hold, less two
// buffers of 1,024 records' metadata and the static shared memory.
constexpr size_t kStagedSmemMax = 232448 - 2 * 1024 * 16 - 512;
// Device status word bits (the word after the work-queue head): a bounded
// wait gave up; a bounds check of the debug build failed.
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint32_t kStatusBounds = 2u;
// Bounds checks of the debug build (GW_DEBUG_BOUNDS): a failed check sets
// kStatusBounds in the status word and the caller skips the access.  In
// the release build the checks compile to `true`.
#ifdef GW_DEBUG_BOUNDS
__device__ __forceinline__ bool gw_in_bounds(bool ok, uint32_t* status) {
    if (!ok && status) atomicOr(status, kStatusBounds);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool gw_in_bounds(bool, uint32_t*) { return true; }
#endif

// Zeroed elements after the last kernel slice of the unpadded tables: the
// staged degridder loads kernel values up to this many elements past a slice.
constexpr int64_t kTableSlack = 256;
int degrid_staged_tile();
bool degrid_staged_fits(int hmax, int npol);
// Returns false (nothing launched) if the region does not fit.
bool launch_degrid_staged(const DegridArgs& a, int hmax, int num_sms, cudaStream_t s);

// ---- full compression (gw_compress.cu) --------------------------------------
struct CompressScratch {
    unsigned long long* keys = nullptr;   // [cap] hash keys (all ones = empty)
    float2* acc = nullptr;                // [cap * npol] summed weighted visibilities
    gw_index_rec* rec = nullptr;          // [chunk] compressed records
    float2* vis = nullptr;                // [chunk * npol] their visibilities
    unsigned long long* count = nullptr;  // [1] compressed records of the current chunk
    unsigned long long* total = nullptr;  // [1] compressed records of the call
    unsigned long long* n_in = nullptr;   // [1] valid records inserted (accumulates)
    int64_t cap = 0;                      // power of two >= 2 * chunk
};
// Adds the weighted visibilities of valid records with equal (k, o, plane,
// sign of w) and writes the distinct records to cs.rec / cs.vis (*cs.count
// of them, order unspecified); the table is left empty for the next call.
void launch_compress(const gw_index_rec* rec, int64_t nvis, const void* vis, int vis_kind,
                     const float* weight, int npol, int beta, CompressScratch& cs,
                     cudaStream_t s);
void clear_compress_table(CompressScratch& cs, int npol, cudaStream_t s);

// ---- hybrid gridding (gw_hybrid.cu) ------------------------------------------
void launch_hybrid_grid(const gw_index_rec* rec, int64_t nvis, const void* vis, int vis_kind,
                        const float* weight, int npol, int beta, int S, const double* c1,
                        int fmin, double norm, int N, int sz, float2* fine,
                        unsigned long long* dropped, cudaStream_t s);
// z: device Z table [beta/2][sz]; h_z: its host copy (null = shared-memory
// tiled pruner only); the streaming pruner covers beta in {8, 16}, sz in 7..15.
void launch_prune(const float2* fine, int npol, int N, int beta, int sz, const float* z,
                  const float* h_z, int num_sms, float2* pruned, cudaStream_t s);
void launch_hybrid_shift(float2* g, int npol, int N, cudaStream_t s);
void launch_hybrid_image(const float2* raw, int npol, int N, const float* hco, const float* hpr,
                         float2* image, cudaStream_t s);

// ---- FP32 FMA throughput probe (gw_peak.cu) ---------------------------------
cudaError_t measure_ffma_peak(int num_sms, int iters, double* tflops, cudaStream_t s);

// ---- allocation-free scratch (gw_noalloc.cu) ------------------------------
// View of the file-scope static scratch on the current device: the symbol's
// device address is looked up on every call (no allocation once the module
// is loaded).
cudaError_t static_scratch_view(Scratch* sc);
// Loads, on the current device, the module holding the static scratch (the
// driver allocates the array then) and every kernel the allocation-free
// degridding path launches for (npol, table_kind), so that its calls need
// no allocation under lazy module loading.
cudaError_t static_path_prepare(int npol, int table_kind);
// Kernel preloading (cudaFuncGetAttributes) of the stages that path uses.
cudaError_t preload_index_kernels();
cudaError_t preload_bin_kernels();
cudaError_t preload_degrid_kernel(int npol, int table_kind);
int64_t static_scratch_max_vis();
int static_scratch_max_tiles();

// ---- correction (gw_correct.cu) -------------------------------------------
void launch_correct(float2* image, const float* h, int N, int npol, int mode, cudaStream_t s);
void launch_shift(float2* grid, int N, int npol, cudaStream_t s);
// image[p][i][j] += sum_l layers[l][p][i][j] exp(+j 2 pi w_l (n_ij - 1)),
// w_l = wmin + l dw, l_j = (j - N/2) cell, m_i = (i - N/2) cell (w-stacking).
void launch_wstack_combine(const float2* layers, int nlayers, double wmin, double dw, int N,
                           int npol, double cell, float2* image, cudaStream_t s);
// grid[i] += err[i]; err[i] = 0 over n complex elements.
void launch_fold(float2* grid, float2* err, int64_t n, cudaStream_t s);
// Zero elements [0, min(n_max, dc count) * npol) of a visibility buffer of kind `kind`.
void launch_zero_vis(void* vis, int kind, int64_t n_max, int npol, DevCount dc, cudaStream_t s);

}  // namespace gw
