// C ABI of libgw: plan lifetime, argument checking, chunking, launches.
// See include/gw.h for the contract of every entry point.
#include "gw_internal.cuh"

#include <mutex>
#include <unordered_map>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace gw {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Allocation-failure injection (gw_debug_fail_alloc): > 0 counts down the
// allocations still allowed to succeed plus one; the allocation that takes
// it from 1 to 0 fails.  0 = off.
static std::atomic<int64_t> g_fail_countdown{0};
static std::atomic<int64_t> g_live_plans{0};

int current_sm_count() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < kMaxDev) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
        return 1;
    if (dev < kMaxDev) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

bool alloc_fault() {
    int64_t k = g_fail_countdown.load();
    while (k > 0) {
        if (g_fail_countdown.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}

// Live device allocations of the library (gw_debug_live_bytes).
static std::mutex g_alloc_mutex;
static std::unordered_map<void*, size_t> g_allocs;
static int64_t g_live_bytes = 0;

cudaError_t dev_alloc(void** ptr, size_t bytes) {
    if (alloc_fault()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        g_allocs[*ptr] = bytes;
        g_live_bytes += (int64_t)bytes;
    }
    return e;
}

void dev_free(void* ptr) {
    if (!ptr) return;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        auto it = g_allocs.find(ptr);
        if (it != g_allocs.end()) {
            g_live_bytes -= (int64_t)it->second;
            g_allocs.erase(it);
        }
    }
    cudaFree(ptr);
}

static thread_local std::string t_last_error;

static gw_status fail(gw_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static gw_status fail(gw_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return st;
}

static gw_status cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? GW_ENOMEM : GW_ECUDA, "%s: %s (%s)", where,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

template <class T>
static T* host_new() {
    return alloc_fault() ? nullptr : new (std::nothrow) T;
}

}  // namespace gw

using namespace gw;

// Device tables of a plan, shared by the plan and its clones (gw_plan_clone);
// freed with the last of them.
struct TableSet {
    std::atomic<int> refs{1};
    float2* table = nullptr;
    uint32_t* table16 = nullptr;
    void* ptable = nullptr;
    int64_t* d_pplane_off = nullptr;
    int64_t* d_plane_off = nullptr;
    int* d_support = nullptr;
    double* d_h = nullptr;
    float* d_hf = nullptr;
    int64_t bytes = 0;
};

struct gw_plan_s {
    gw_plan_desc desc{};
    int device = -1;
    int num_sms = 0;
    BinGeom geom_grid{}, geom_degrid{}, geom_staged{};
    int hmax = 0;        // largest half-support over the planes
    int ntiles = 0;      // bins allocated (max over the geometries and plane groups)
    int max_groups = 1;  // plane groups the bins are allocated for (gw_tuning.plane_groups)
    int auto_groups = 1; // plane groups chosen when plane_groups = 0
    int pad_stride = 0;
    double field = 0, table_scale = 0;
    std::vector<int> support;
    std::vector<double> wplane;
    std::vector<int64_t> plane_off;
    int max_tiles_per_vis = 0;
    int64_t chunk = 0;
    TableSet* tabs = nullptr;     // owner of the device tables below once the plan is built
    CompressScratch cs;           // full-compression scratch (allocated on first use)
    // w-stacking bins over layers x tiles (allocated on first use, grown on demand)
    int ws_layers = 0;
    uint32_t *ws_count = nullptr, *ws_offsets = nullptr, *ws_cursor = nullptr,
             *ws_item_off = nullptr;
    Item* ws_items = nullptr;
    int64_t ws_items_cap = 0;
    // hybrid gridding: the 1-D w = 0 kernel (kept from the table build) and
    // the pruner of the last support used
    double* d_c1 = nullptr;
    int c1_fmin = 0;
    double c1_norm = 1.0;
    // host-input pipeline (gw_grid_vis_host): a copy stream, two staging sets
    cudaStream_t h_copy = nullptr;
    // banded read-back (gw_grid_vis_devcount_readback): copy stream and
    // per-band events, created on first use
    cudaStream_t rb_stream = nullptr;
    std::vector<cudaEvent_t> rb_ev;
    cudaEvent_t h_ready[2] = {nullptr, nullptr}, h_free[2] = {nullptr, nullptr};
    double* h_uvw[2] = {nullptr, nullptr};
    void* h_vis[2] = {nullptr, nullptr};
    float* h_wt[2] = {nullptr, nullptr};
    double* h_freq = nullptr;
    int64_t h_rows = 0, h_freq_n = 0;
    int hy_sz = 0;
    float* d_z = nullptr;
    std::vector<float> h_z;       // host copy of d_z (kernel-argument weights)
    double* d_hpr = nullptr;
    float* d_hprf = nullptr;
    int64_t scratch_bytes = 0;
    gw_tuning tuning{};
    // device state
    float2* table = nullptr;      // FP32 tables (always built)
    uint32_t* table16 = nullptr;  // 16-bit-pair tables (table_dtype != GW_C64)
    void* ptable = nullptr;       // zero-padded gridder tables of kind grid_tk
    int grid_tk = GW_C64;         // their kind: table_dtype, or kTabRealF32 (w = 0 kernel)
    int table_exp2 = 0;           // 16-bit tables hold K * 2^table_exp2
    float table_inv = 1.f;        // 2^-table_exp2
    std::vector<int64_t> pplane_off;
    int64_t* d_pplane_off = nullptr;
    int64_t* d_plane_off = nullptr;
    int* d_support = nullptr;
    double* d_h = nullptr;
    float* d_hf = nullptr;
    Scratch sc;
    IndexParams ip{};
    // tracing
    bool timing = false;
    struct Ev { int stage; cudaEvent_t a, b; };
    std::vector<Ev> events;
    std::vector<cudaEvent_t> pool;
};

namespace {

void free_tables(float2* table, uint32_t* table16, void* ptable, int64_t* d_pplane_off,
                 int64_t* d_plane_off, int* d_support, double* d_h, float* d_hf) {
    dev_free(table);
    dev_free(table16);
    dev_free(ptable);
    dev_free(d_pplane_off);
    dev_free(d_plane_off);
    dev_free(d_support);
    dev_free(d_h);
    dev_free(d_hf);
}

void plan_free(gw_plan p) {
    if (!p) return;
    for (auto& e : p->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (auto e : p->pool) cudaEventDestroy(e);
    dev_free(p->sc.work);
    dev_free(p->sc.wvis);
    dev_free(p->cs.keys);
    dev_free(p->cs.acc);
    dev_free(p->cs.rec);
    dev_free(p->cs.vis);
    dev_free(p->cs.count);
    dev_free(p->ws_count);
    dev_free(p->ws_offsets);
    dev_free(p->ws_cursor);
    dev_free(p->ws_item_off);
    dev_free(p->ws_items);
    for (int b = 0; b < 2; ++b) {
        dev_free(p->h_uvw[b]);
        dev_free(p->h_vis[b]);
        dev_free(p->h_wt[b]);
        if (p->h_ready[b]) cudaEventDestroy(p->h_ready[b]);
        if (p->h_free[b]) cudaEventDestroy(p->h_free[b]);
    }
    dev_free(p->h_freq);
    if (p->h_copy) cudaStreamDestroy(p->h_copy);
    for (auto ev : p->rb_ev) cudaEventDestroy(ev);
    if (p->rb_stream) cudaStreamDestroy(p->rb_stream);
    dev_free(p->d_c1);
    dev_free(p->d_z);
    dev_free(p->d_hpr);
    dev_free(p->d_hprf);
    if (p->tabs) {
        TableSet* t = p->tabs;
        if (t->refs.fetch_sub(1) == 1) {
            free_tables(t->table, t->table16, t->ptable, t->d_pplane_off, t->d_plane_off,
                        t->d_support, t->d_h, t->d_hf);
            delete t;
        }
    } else {   // a plan that failed before its tables were handed to a TableSet
        free_tables(p->table, p->table16, p->ptable, p->d_pplane_off, p->d_plane_off,
                    p->d_support, p->d_h, p->d_hf);
    }
    dev_free(p->sc.rec);
    dev_free(p->sc.count);
    dev_free(p->sc.offsets);
    dev_free(p->sc.cursor);
    dev_free(p->sc.item_off);
    dev_free(p->sc.entries);
    dev_free(p->sc.items);
    dev_free(p->sc.scan_tmp);
    dev_free(p->sc.counters);
    dev_free(p->sc.dropped);
    delete p;
}

gw_status check_desc(const gw_plan_desc* d) {
    if (!d) return fail(GW_EINVAL, "null descriptor");
    if (d->grid_n < 8 || d->grid_n > 32768 || (d->grid_n & 1))
        return fail(GW_EINVAL, "grid_n must be even and in [8, 32768] (got %d)", d->grid_n);
    if (!(d->cell_rad > 0.0) || !std::isfinite(d->cell_rad))
        return fail(GW_EINVAL, "cell_rad must be positive and finite");
    if (d->support_min < 1 || !(d->support_min & 1) || d->support_max < d->support_min ||
        !(d->support_max & 1) || d->support_max > 255)
        return fail(GW_EINVAL, "supports must be odd with 1 <= support_min <= support_max <= 255");
    if (d->oversample < 2 || d->oversample > 256 || (d->oversample & 1))
        return fail(GW_EINVAL, "oversample must be even and in [2, 256]");
    if (d->n_wplanes < 1 || d->n_wplanes > 4096)
        return fail(GW_EINVAL, "n_wplanes must be in [1, 4096]");
    if (d->npol < 1 || d->npol > 4) return fail(GW_EINVAL, "npol must be in [1, 4]");
    if (d->n_wplanes > 1 && !(d->w_max_lambda > 0.0 && std::isfinite(d->w_max_lambda)))
        return fail(GW_EINVAL, "w_max_lambda must be positive when n_wplanes > 1");
    const double half = 0.5 * d->grid_n * d->cell_rad;
    if (d->n_wplanes > 1 && 2.0 * half * half >= 1.0)
        return fail(GW_EINVAL, "field of view too wide: corners reach l^2 + m^2 >= 1");
    if (d->vis_dtype < GW_C64 || d->vis_dtype > GW_F16X2)
        return fail(GW_EINVAL, "vis_dtype must be GW_C64, GW_BF16X2 or GW_F16X2");
    if (d->table_dtype < GW_C64 || d->table_dtype > GW_F16X2)
        return fail(GW_EINVAL, "table_dtype must be GW_C64, GW_BF16X2 or GW_F16X2");
    if (d->max_vis_per_call < 0) return fail(GW_EINVAL, "max_vis_per_call must be >= 0");
    return GW_OK;
}

gw_status check_device(gw_plan p) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(GW_EDEVICE, "plan lives on device %d but device %d is current", p->device, dev);
    return GW_OK;
}

template <class T>
cudaError_t dmalloc(T** ptr, size_t n) {
    return dev_alloc((void**)ptr, sizeof(T) * (n ? n : 1));
}

// Per-plan scratch sized by the plan's chunk (gw_plan_clone gives each clone its own).
gw_status alloc_scratch(gw_plan p) {
    Scratch& sc = p->sc;
    sc.entries_cap = p->chunk * p->max_tiles_per_vis;
    sc.items_cap = sc.entries_cap / kItemMin + p->ntiles + 1;
    cudaError_t e = cudaSuccess;
    int64_t bytes = 0;
#define GW_ALLOC(x, n) do { e = dmalloc(&(x), (n)); \
        if (e != cudaSuccess) return fail(GW_ENOMEM, "device allocation of %s failed", #x); \
        bytes += (int64_t)sizeof(*(x)) * (int64_t)(n); } while (0)
    GW_ALLOC(sc.rec, (size_t)p->chunk);
    GW_ALLOC(sc.count, (size_t)p->ntiles);
    GW_ALLOC(sc.offsets, (size_t)p->ntiles + 1);
    GW_ALLOC(sc.cursor, (size_t)p->ntiles);
    GW_ALLOC(sc.item_off, (size_t)p->ntiles + 1);
    GW_ALLOC(sc.entries, (size_t)sc.entries_cap);
    GW_ALLOC(sc.items, (size_t)sc.items_cap);
    GW_ALLOC(sc.scan_tmp, (size_t)scan_tmp_words(p->ntiles));
    sc.scan_tmp_bins = p->ntiles;
    GW_ALLOC(sc.counters, 4);
    GW_ALLOC(sc.dropped, 1);
    GW_ALLOC(sc.work, 2);
#undef GW_ALLOC
    p->scratch_bytes = bytes;
    // counters[1] is the device status word (a bounded device wait gave up)
    e = cudaMemset(sc.counters, 0, 4 * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "clearing the device status word");
    return GW_OK;
}

// Work-item size and degridding kernel choice of a plan (gw_plan_set_tuning).
void apply_tuning(gw_plan p) {
    const int im = p->tuning.item_max > 0 ? p->tuning.item_max : kItemMax;
    p->geom_grid.item_max = im;
    p->geom_degrid.item_max = im;
    p->geom_staged.item_max = im;
}

enum Stage { kStIndex = 0, kStBin = 1, kStGrid = 2, kStDegrid = 3 };

cudaEvent_t take_event(gw_plan p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets one stage with CUDA events on the launch stream when timing is on.
struct StageTimer {
    gw_plan p;
    cudaStream_t s;
    int stage;
    cudaEvent_t a = nullptr;
    StageTimer(gw_plan p_, int stage_, cudaStream_t s_) : p(p_), s(s_), stage(stage_) {
        if (p->timing && (a = take_event(p))) cudaEventRecord(a, s);
    }
    ~StageTimer() {
        if (!a) return;
        cudaEvent_t b = take_event(p);
        if (!b) { p->pool.push_back(a); return; }
        cudaEventRecord(b, s);
        p->events.push_back({stage, a, b});
    }
};

// Index + bin one chunk of rows; leaves records and bins in the plan scratch.
gw_status index_and_bin(gw_plan p, const double* uvw, const double* freq, int64_t nrow, int nchan,
                        const BinGeom& geom, cudaStream_t s) {
    {
        StageTimer t(p, kStIndex, s);
        launch_index(uvw, freq, nrow, nchan, p->ip, p->sc.rec, p->sc.dropped, s);
    }
    {
        StageTimer t(p, kStBin, s);
        launch_bin(p->sc.rec, nrow * (int64_t)nchan, geom, p->desc.n_wplanes,
                   p->desc.support_min, p->desc.support_max, p->sc, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "index/bin launch");
    return GW_OK;
}

int64_t rows_per_chunk(gw_plan p, int nchan) {
    int64_t r = p->chunk / (nchan > 0 ? nchan : 1);
    return r < 1 ? 1 : r;
}

// Reads (and clears) the plan's device status word; the stream must have
// been synchronised.  GW_ETIMEDOUT when a bounded device wait gave up.
gw_status read_device_status(gw_plan p) {
    uint32_t st = 0;
    cudaError_t e = cudaMemcpy(&st, p->sc.counters + 1, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
    if (st == 0) return GW_OK;
    e = cudaMemset(p->sc.counters + 1, 0, sizeof st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the device status word");
    if (st & kStatusBounds)
        return fail(GW_EBOUNDS, "a device bounds check failed (status 0x%x); the results of the "
                    "calls since the last check are wrong", st);
    return fail(GW_ETIMEDOUT, "a bounded device wait gave up (status 0x%x); the results of the "
                "calls since the last check are incomplete", st);
}

gw_status finish_dropped(gw_plan p, int64_t* n_dropped, cudaStream_t s) {
    if (!n_dropped) return GW_OK;
    unsigned long long h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p->sc.dropped, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the drop count");
    *n_dropped = (int64_t)h;
    return read_device_status(p);
}

gw_status common_checks(gw_plan p, const double* uvw, const double* freq, int64_t nrow, int nchan) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    if (nrow < 0 || nchan < 0) return fail(GW_EINVAL, "negative nrow or nchan");
    if (nrow > 0 && nchan > 0 && (!uvw || !freq)) return fail(GW_EINVAL, "null uvw or freq");
    if ((int64_t)nchan > p->chunk)
        return fail(GW_EINVAL, "nchan (%d) exceeds the plan's chunk size", nchan);
    return GW_OK;
}

}  // namespace

extern "C" {

int32_t gw_api_version(void) { return GW_API_VERSION; }

uint64_t gw_launch_count(void) { return g_launches.load(); }

const char* gw_strerror(gw_status s) {
    switch (s) {
        case GW_OK: return "success";
        case GW_EINVAL: return "invalid argument";
        case GW_ENOMEM: return "out of memory";
        case GW_ECUDA: return "CUDA error";
        case GW_ETIMEDOUT: return "device wait timed out";
        case GW_EUNSUPPORTED: return "unsupported";
        case GW_EDEVICE: return "wrong current device";
        case GW_EBOUNDS: return "device bounds check failed";
    }
    return "unknown status";
}

const char* gw_last_error(void) { return t_last_error.c_str(); }

gw_status gw_plan_create(const gw_plan_desc* desc, void* cuda_stream, gw_plan* out) {
    if (!out) return fail(GW_EINVAL, "null output pointer");
    *out = nullptr;
    gw_status st = check_desc(desc);
    if (st != GW_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    gw_plan p = host_new<gw_plan_s>();
    if (!p) return fail(GW_ENOMEM, "host allocation failed");
    p->desc = *desc;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "cudaGetDevice"); }
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "cudaDeviceGetAttribute"); }

    const int N = desc->grid_n, P = desc->n_wplanes, beta = desc->oversample;
    p->field = (double)N * desc->cell_rad;
    p->geom_grid = BinGeom{0, kGridTileShiftU, 5, (N + kGridTileU - 1) / kGridTileU,
                           (N + kGridTileV - 1) / kGridTileV};
    p->geom_degrid = BinGeom{1, 5, 5, (N + kTile - 1) / kTile, (N + kTile - 1) / kTile};
    {
        const int st = degrid_staged_tile();
        p->geom_staged = BinGeom{1, 4, 4, (N + st - 1) / st, (N + st - 1) / st};
    }
    p->ntiles = std::max({p->geom_grid.ntu * p->geom_grid.ntv,
                          p->geom_degrid.ntu * p->geom_degrid.ntv,
                          p->geom_staged.ntu * p->geom_staged.ntv});
    p->support.resize(P);
    p->wplane.resize(P);
    p->plane_off.resize(P + 1);
    p->plane_off[0] = 0;
    p->pplane_off.resize(P + 1);
    p->pplane_off[0] = 0;
    int smax_real = 0;
    for (int q = 0; q < P; ++q) {
        p->support[q] = plane_support(q, P, desc->support_min, desc->support_max);
        smax_real = std::max(smax_real, p->support[q]);
    }
    p->pad_stride = padded_stride(smax_real);
    p->hmax = smax_real / 2;
    for (int q = 0; q < P; ++q) {
        const double r = P > 1 ? (double)q / (double)(P - 1) : 0.0;
        p->wplane[q] = P > 1 ? desc->w_max_lambda * (r * r) : 0.0;
        p->plane_off[q + 1] = p->plane_off[q] + (int64_t)beta * beta * p->support[q] * p->support[q];
        p->pplane_off[q + 1] = p->pplane_off[q] + padded_table_elems(p->support[q], beta, p->pad_stride);
    }
    if (p->pplane_off[P] >= (int64_t)1 << 31) {
        plan_free(p);
        return fail(GW_EINVAL, "kernel tables exceed 2^31 elements");
    }
    // plane groups: bins keyed by (group of consecutive w-planes, tile) keep
    // one group's padded tables in L2 while its items are gridded; chosen
    // automatically for FP32 tables above kGroupTableBytes (16-bit tables
    // did not grid faster in groups, and grouped binning costs more)
    p->max_groups = P > 1 ? std::min(P, kMaxPlaneGroups) : 1;
    {
        const int64_t tb = p->pplane_off[P] * (int64_t)dtype_bytes(desc->table_dtype);
        const int64_t g = desc->table_dtype == GW_C64 && tb > kGroupTableBytes
                              ? (tb + kGroupTargetBytes - 1) / kGroupTargetBytes : 1;
        p->auto_groups = (int)std::min<int64_t>(g, p->max_groups);
    }
    p->ntiles = std::max(p->ntiles, p->geom_grid.ntu * p->geom_grid.ntv * p->max_groups);
    p->max_tiles_per_vis = std::max(((smax_real - 1) / kGridTileU + 2) * ((smax_real - 1) / kGridTileV + 2), 1);
    p->chunk = desc->max_vis_per_call > 0 ? desc->max_vis_per_call : ((int64_t)1 << 23);
    if (p->chunk * p->max_tiles_per_vis >= ((int64_t)1 << 32)) {
        plan_free(p);
        return fail(GW_EINVAL, "max_vis_per_call too large for 32-bit bin entries");
    }

    p->ip.L = p->field;
    p->ip.halfN = (double)(N / 2);
    p->ip.beta_d = (double)beta;
    p->ip.Pm1_d = (double)(P - 1);
    p->ip.wmax = desc->w_max_lambda;
    p->ip.N = N;
    p->ip.beta = beta;
    p->ip.P = P;
    p->ip.smin = desc->support_min;
    p->ip.smax = desc->support_max;

#define GW_ALLOC(x, n) do { e = dmalloc(&(x), (n)); if (e != cudaSuccess) { plan_free(p); \
        return fail(GW_ENOMEM, "device allocation of %s failed", #x); } } while (0)
    GW_ALLOC(p->table, (size_t)(p->plane_off[P] + kTableSlack));
    // 2-D plans (P = 1) grid with the real w = 0 kernel: its imaginary parts
    // are exactly zero, so the gridder's padded table keeps the real parts
    p->grid_tk = desc->table_dtype == GW_C64 && P == 1 ? kTabRealF32 : desc->table_dtype;
    if (p->grid_tk == kTabRealF32) {
        float* pt = nullptr;
        GW_ALLOC(pt, (size_t)p->pplane_off[P]);
        p->ptable = pt;
    } else if (desc->table_dtype == GW_C64) {
        float2* pt = nullptr;
        GW_ALLOC(pt, (size_t)p->pplane_off[P]);
        p->ptable = pt;
    } else {
        uint32_t* pt = nullptr;
        GW_ALLOC(p->table16, (size_t)(p->plane_off[P] + kTableSlack));
        GW_ALLOC(pt, (size_t)p->pplane_off[P]);
        p->ptable = pt;
    }
    // the slack after the last slice reads as zeros
    e = cudaMemset(p->table + p->plane_off[P], 0, sizeof(float2) * kTableSlack);
    if (e == cudaSuccess && p->table16)
        e = cudaMemset(p->table16 + p->plane_off[P], 0, sizeof(uint32_t) * kTableSlack);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaMemset");
    }
    GW_ALLOC(p->d_pplane_off, (size_t)P + 1);
    GW_ALLOC(p->d_plane_off, (size_t)P + 1);
    GW_ALLOC(p->d_support, (size_t)P);
    GW_ALLOC(p->d_h, (size_t)N);
    GW_ALLOC(p->d_hf, (size_t)N);
    GW_ALLOC(p->d_c1, (size_t)beta * p->support[0]);
#undef GW_ALLOC
    if (alloc_scratch(p) != GW_OK) {
        plan_free(p);
        return GW_ENOMEM;
    }
    Scratch& sc = p->sc;
    e = cudaMemsetAsync(sc.work, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "cudaMemsetAsync"); }
    e = cudaMemcpyAsync(p->d_plane_off, p->plane_off.data(), sizeof(int64_t) * (P + 1),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_pplane_off, p->pplane_off.data(), sizeof(int64_t) * (P + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_support, p->support.data(), sizeof(int) * P,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "uploading plane metadata"); }

    TableBuild tb;
    tb.N = N;
    tb.beta = beta;
    tb.P = P;
    tb.smin = desc->support_min;
    tb.smax = desc->support_max;
    tb.field = p->field;
    tb.wmax = desc->w_max_lambda;
    tb.support = p->support.data();
    tb.wplane = p->wplane.data();
    tb.plane_off = p->plane_off.data();
    tb.num_sms = p->num_sms;
    e = build_tables(tb, p->table, p->table16, desc->table_dtype, p->d_h, p->d_hf,
                     &p->table_scale, &p->table_exp2, p->d_c1, s);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "building kernel tables"); }
    {
        // normalisation of the 1-D kernel: its zero-offset taps sum to 1
        const int S0 = p->support[0], h0 = S0 / 2;
        p->c1_fmin = -beta * h0 - beta / 2 + 1;
        std::vector<double> c1((size_t)beta * S0);
        e = cudaMemcpy(c1.data(), p->d_c1, sizeof(double) * c1.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "reading the 1-D kernel"); }
        double nrm = 0.0;
        for (int t = -h0; t <= h0; ++t) nrm += c1[beta * t - p->c1_fmin];
        p->c1_norm = nrm;
    }
    p->table_inv = std::ldexp(1.0f, -p->table_exp2);
    if (desc->table_dtype == GW_C64)
        launch_pad_tables(p->table, p->grid_tk, p->d_plane_off, p->d_pplane_off, p->d_support, P,
                          beta, p->pad_stride, p->ptable, s);
    else
        launch_pad_tables(p->table16, desc->table_dtype, p->d_plane_off, p->d_pplane_off,
                          p->d_support, P, beta, p->pad_stride, p->ptable, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "padding kernel tables"); }
    TableSet* t = host_new<TableSet>();
    if (!t) { plan_free(p); return fail(GW_ENOMEM, "host allocation failed"); }
    t->table = p->table;
    t->table16 = p->table16;
    t->ptable = p->ptable;
    t->d_pplane_off = p->d_pplane_off;
    t->d_plane_off = p->d_plane_off;
    t->d_support = p->d_support;
    t->d_h = p->d_h;
    t->d_hf = p->d_hf;
    t->bytes = (int64_t)sizeof(float2) * (p->plane_off[P] + kTableSlack) +
               (int64_t)(p->grid_tk == kTabRealF32 ? sizeof(float) : dtype_bytes(desc->table_dtype)) *
                   p->pplane_off[P] +
               (p->table16 ? (int64_t)sizeof(uint32_t) * (p->plane_off[P] + kTableSlack) : 0) +
               (int64_t)(2 * sizeof(int64_t) + sizeof(int)) * (P + 1) +
               (int64_t)(sizeof(double) + sizeof(float)) * N;
    p->tabs = t;
    // the allocation-free degridding path allocates nothing when called: its
    // module (static scratch) and kernels are loaded now, while allocating is
    // still allowed
    e = static_path_prepare(desc->npol, desc->table_dtype);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "loading the allocation-free path"); }
    apply_tuning(p);
    g_live_plans.fetch_add(1);
    *out = p;
    return GW_OK;
}

gw_status gw_plan_clone(gw_plan src, int64_t max_vis_per_call, void* cuda_stream, gw_plan* out) {
    if (!out) return fail(GW_EINVAL, "null output pointer");
    *out = nullptr;
    if (!src || !src->tabs) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(src);
    if (st != GW_OK) return st;
    if (max_vis_per_call < 0) return fail(GW_EINVAL, "max_vis_per_call must be >= 0");
    gw_plan p = host_new<gw_plan_s>();
    if (!p) return fail(GW_ENOMEM, "host allocation failed");
    p->desc = src->desc;
    p->desc.max_vis_per_call = max_vis_per_call;
    p->device = src->device;
    p->num_sms = src->num_sms;
    p->geom_grid = src->geom_grid;
    p->geom_degrid = src->geom_degrid;
    p->geom_staged = src->geom_staged;
    p->hmax = src->hmax;
    p->ntiles = src->ntiles;
    p->max_groups = src->max_groups;
    p->auto_groups = src->auto_groups;
    p->pad_stride = src->pad_stride;
    p->field = src->field;
    p->table_scale = src->table_scale;
    p->support = src->support;
    p->wplane = src->wplane;
    p->plane_off = src->plane_off;
    p->pplane_off = src->pplane_off;
    p->max_tiles_per_vis = src->max_tiles_per_vis;
    p->ip = src->ip;
    p->tuning = src->tuning;
    p->chunk = max_vis_per_call > 0 ? max_vis_per_call : ((int64_t)1 << 23);
    if (p->chunk * p->max_tiles_per_vis >= ((int64_t)1 << 32)) {
        delete p;
        return fail(GW_EINVAL, "max_vis_per_call too large for 32-bit bin entries");
    }
    // share the tables
    p->tabs = src->tabs;
    p->tabs->refs.fetch_add(1);
    p->table = src->table;
    p->table16 = src->table16;
    p->ptable = src->ptable;
    p->grid_tk = src->grid_tk;
    p->table_exp2 = src->table_exp2;
    p->table_inv = src->table_inv;
    p->d_pplane_off = src->d_pplane_off;
    p->d_plane_off = src->d_plane_off;
    p->d_support = src->d_support;
    p->d_h = src->d_h;
    p->d_hf = src->d_hf;
    st = alloc_scratch(p);
    if (st != GW_OK) { plan_free(p); return st; }
    p->c1_fmin = src->c1_fmin;
    p->c1_norm = src->c1_norm;
    const size_t nc1 = (size_t)src->desc.oversample * src->support[0];
    cudaError_t e = dmalloc(&p->d_c1, nc1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_c1, src->d_c1, sizeof(double) * nc1, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "copying the 1-D kernel"); }
    e = cudaMemsetAsync(p->sc.work, 0, 2 * sizeof(unsigned long long),
                        (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e, "cudaMemsetAsync"); }
    apply_tuning(p);
    g_live_plans.fetch_add(1);
    *out = p;
    return GW_OK;
}

gw_status gw_plan_set_tuning(gw_plan p, const gw_tuning* t) {
    if (!p || !t) return fail(GW_EINVAL, "null argument");
    if (t->item_max != 0 && (t->item_max < kItemMin || t->item_max > (1 << 20)))
        return fail(GW_EINVAL, "item_max must be 0 or in [%d, 2^20]", kItemMin);
    if (t->degrid_kernel < 0 || t->degrid_kernel > 2)
        return fail(GW_EINVAL, "degrid_kernel must be 0 (auto), 1 (staged) or 2 (gather)");
    if (t->grid_kernel < 0 || t->grid_kernel > 2)
        return fail(GW_EINVAL, "grid_kernel must be 0 (auto), 1 (binned) or 2 (direct)");
    if (t->compress_min_gain < 0 || t->compress_min_gain > 1000)
        return fail(GW_EINVAL, "compress_min_gain must be in [0, 1000] (per mille)");
    if (t->plane_groups < 0 || t->plane_groups > p->max_groups)
        return fail(GW_EINVAL, "plane_groups must be in [0, %d] for this plan", p->max_groups);
    p->tuning = *t;
    apply_tuning(p);
    return GW_OK;
}

gw_status gw_plan_get_tuning(gw_plan p, gw_tuning* out) {
    if (!p || !out) return fail(GW_EINVAL, "null argument");
    *out = p->tuning;
    return GW_OK;
}

gw_status gw_plan_device_status(gw_plan p, void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return read_device_status(p);
}

gw_status gw_plan_destroy(gw_plan plan) {
    if (plan) g_live_plans.fetch_sub(1);
    plan_free(plan);
    return GW_OK;
}

gw_status gw_debug_fail_alloc(int64_t n) {
    if (n < 0) return fail(GW_EINVAL, "n must be >= 0");
    g_fail_countdown.store(n);
    return GW_OK;
}

int64_t gw_debug_live_plans(void) { return g_live_plans.load(); }

int64_t gw_debug_live_bytes(void) {
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    return g_live_bytes;
}

// Plane groups of the binned gridder (gw_tuning.plane_groups, 0 = the plan's
// automatic choice), and the bin geometry for them.
static int grid_groups(gw_plan p) {
    const int g = p->tuning.plane_groups > 0 ? p->tuning.plane_groups : p->auto_groups;
    return std::max(1, std::min(g, p->max_groups));
}
static BinGeom grid_geom(gw_plan p, int groups) {
    BinGeom g = p->geom_grid;
    if (groups > 1) {
        g.layer_tiles = g.ntu * g.ntv;
        g.nlayers = groups;
        g.group_planes = (p->desc.n_wplanes + groups - 1) / groups;
    }
    return g;
}

gw_status gw_plan_info_get(gw_plan p, gw_plan_info* out) {
    if (!p || !out) return fail(GW_EINVAL, "null argument");
    out->grid_n = p->desc.grid_n;
    out->npol = p->desc.npol;
    out->oversample = p->desc.oversample;
    out->n_wplanes = p->desc.n_wplanes;
    out->grid_tile_u = kGridTileU;
    out->grid_tile_v = kGridTileV;
    out->degrid_tile = kTile;
    out->device = p->device;
    out->table_elems = p->plane_off.back();
    out->chunk_vis = p->chunk;
    out->field = p->field;
    out->taper_c = M_PI * p->desc.support_min / 2.0;
    out->table_scale = p->table_scale;
    out->vis_dtype = p->desc.vis_dtype;
    out->table_dtype = p->desc.table_dtype;
    out->table_exp2 = p->table_exp2;
    out->plane_groups = grid_groups(p);
    out->table_bytes = p->tabs ? p->tabs->bytes : 0;
    out->scratch_bytes = p->scratch_bytes;
    return GW_OK;
}

// Direct (unbinned) gridding of a chunk of nvis visibilities: forced by the
// tuning, or automatic for inputs small enough that launches dominate.
static bool use_direct(gw_plan p, int64_t nvis) {
    if (p->tuning.grid_kernel == 1) return false;
    if (p->tuning.grid_kernel == 2) return true;
    const int64_t smax = p->support.empty() ? 1 : p->support.back();
    return nvis <= kDirectMaxVis && nvis * smax * smax * p->desc.npol <= kDirectMaxTaps;
}

static gw_status grid_impl(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                           int32_t nchan, const void* vis, const float* weight, void* grid,
                           void* grid_err, int64_t* n_dropped, void* cuda_stream,
                           bool reset_dropped = true) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (!grid) return fail(GW_EINVAL, "null grid");
    if (nrow > 0 && nchan > 0 && !vis) return fail(GW_EINVAL, "null vis");
    const int vk = p->desc.vis_dtype;
    const size_t vb = dtype_bytes(vk);
    if (vk == GW_C64 && (p->desc.npol % 2 == 0) && (reinterpret_cast<uintptr_t>(vis) % 16 != 0))
        return fail(GW_EINVAL, "vis must be 16-byte aligned when npol is even");
    if ((reinterpret_cast<uintptr_t>(grid) % 8 != 0) || (reinterpret_cast<uintptr_t>(vis) % vb != 0))
        return fail(GW_EINVAL, "grid must be 8-byte aligned and vis aligned to its element size");
    if (grid_err && reinterpret_cast<uintptr_t>(grid_err) % 8 != 0)
        return fail(GW_EINVAL, "grid_err must be 8-byte aligned");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = reset_dropped ? cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s)
                                  : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const int npol = p->desc.npol;
    const int64_t rpc = rows_per_chunk(p, nchan);
    for (int64_t r0 = 0; r0 < nrow && nchan > 0; r0 += rpc) {
        const int64_t nr = std::min(rpc, nrow - r0);
        const int64_t v0 = r0 * nchan;
        if (use_direct(p, nr * nchan)) {
            // small input: one launch that indexes and grids (weights applied
            // in the kernel)
            GridArgs a;
            a.rec = nullptr;
            a.vis = static_cast<const char*>(vis) + (size_t)v0 * npol * vb;
            a.vis_kind = vk;
            a.weight = weight ? weight + v0 * npol : nullptr;
            a.table_kind = p->desc.table_dtype;
            a.table_inv = p->table_inv;
            a.plane_off = p->d_plane_off;
            a.support = p->d_support;
            a.grid = reinterpret_cast<float2*>(grid);
            a.grid_err = reinterpret_cast<float2*>(grid_err);
            a.N = p->desc.grid_n;
            a.npol = npol;
            a.beta = p->desc.oversample;
            {
                StageTimer t(p, kStGrid, s);
                a.queue = p->sc.counters;
                a.table_elems = p->plane_off.back();
                const DirectIndex di{uvw_m + 3 * r0, freq_hz, nr, nchan, p->ip, p->sc.dropped};
                launch_grid_direct(a, p->table16 ? (const void*)p->table16 : (const void*)p->table,
                                   di, p->sc.work, s);
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "grid launch");
            continue;
        }
        const int groups = grid_groups(p);
        const BinGeom geom = grid_geom(p, groups);
        st = index_and_bin(p, uvw_m + 3 * r0, freq_hz, nr, nchan, geom, s);
        if (st != GW_OK) return st;
        GridArgs a;
        a.rec = p->sc.rec;
        a.ptable = p->ptable;
        a.pplane_off = p->d_pplane_off;
        a.vis = static_cast<const char*>(vis) + (size_t)v0 * npol * vb;
        a.vis_kind = vk;
        a.weight = nullptr;
        if (weight) {
            if (!p->sc.wvis) {
                e = dev_alloc((void**)&p->sc.wvis, sizeof(float2) * (size_t)p->chunk * npol);
                if (e != cudaSuccess) {
                    p->sc.wvis = nullptr;
                    return fail(GW_ENOMEM, "allocating weighted-visibility scratch");
                }
            }
            // weighted visibilities are formed in FP32
            launch_weight_vis(a.vis, vk, weight + v0 * npol, nr * nchan * npol, p->sc.wvis, s);
            a.vis = p->sc.wvis;
            a.vis_kind = GW_C64;
        }
        a.table_kind = p->grid_tk;
        a.table_inv = p->table_inv;
        a.plane_off = p->d_plane_off;
        a.support = p->d_support;
        a.entries = p->sc.entries;
        a.items = p->sc.items;
        a.item_count = p->sc.item_off + p->geom_grid.ntu * p->geom_grid.ntv * groups;
        if (groups > 1) {
            a.layer_tiles = p->geom_grid.ntu * p->geom_grid.ntv;
            a.layer_stride = 0;
            a.plane_groups = 1;
        }
        a.queue = p->sc.counters;
        a.grid = reinterpret_cast<float2*>(grid);
        a.grid_err = reinterpret_cast<float2*>(grid_err);
        a.N = p->desc.grid_n;
        a.npol = npol;
        a.beta = p->desc.oversample;
        a.ntiles_u = p->geom_grid.ntu;
        a.pad_stride = p->pad_stride;
        a.ptable_elems = p->pplane_off.back();
        {
            StageTimer t(p, kStGrid, s);
            launch_grid(a, p->num_sms, s);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "grid launch");
    }
    return finish_dropped(p, n_dropped, s);
}

gw_status gw_grid_vis(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                      int32_t nchan, const void* vis, const float* weight, void* grid,
                      int64_t* n_dropped, void* cuda_stream) {
    return grid_impl(p, uvw_m, freq_hz, nrow, nchan, vis, weight, grid, nullptr, n_dropped,
                     cuda_stream);
}

// Staging for the host-input pipeline: two sets of `rows` rows.
static gw_status ensure_host_pipe(gw_plan p, int64_t rows, int nchan) {
    const int npol = p->desc.npol;
    const size_t vb = dtype_bytes(p->desc.vis_dtype);
    cudaError_t e = cudaSuccess;
    if (!p->h_copy) {
        e = cudaStreamCreateWithFlags(&p->h_copy, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&p->h_ready[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->h_free[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "creating the copy stream");
    }
    if (p->h_rows < rows || p->h_freq_n < nchan) {
        for (int b = 0; b < 2; ++b) {
            dev_free(p->h_uvw[b]);
            dev_free(p->h_vis[b]);
            dev_free(p->h_wt[b]);
            p->h_uvw[b] = nullptr;
            p->h_vis[b] = nullptr;
            p->h_wt[b] = nullptr;
        }
        dev_free(p->h_freq);
        p->h_freq = nullptr;
        p->h_rows = 0;
        const int64_t r = std::max(rows, p->h_rows), c = std::max<int64_t>(nchan, p->h_freq_n);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = dev_alloc((void**)&p->h_uvw[b], sizeof(double) * 3 * r);
            if (e == cudaSuccess) e = dev_alloc(&p->h_vis[b], vb * r * c * npol);
            if (e == cudaSuccess) e = dev_alloc((void**)&p->h_wt[b], sizeof(float) * r * c * npol);
        }
        if (e == cudaSuccess) e = dev_alloc((void**)&p->h_freq, sizeof(double) * c);
        if (e != cudaSuccess) {
            // leave no partial staging behind: the next call starts afresh
            for (int b = 0; b < 2; ++b) {
                dev_free(p->h_uvw[b]);
                dev_free(p->h_vis[b]);
                dev_free(p->h_wt[b]);
                p->h_uvw[b] = nullptr;
                p->h_vis[b] = nullptr;
                p->h_wt[b] = nullptr;
            }
            dev_free(p->h_freq);
            p->h_freq = nullptr;
            return fail(GW_ENOMEM, "allocating host-pipeline staging");
        }
        p->h_rows = r;
        p->h_freq_n = c;
    }
    return GW_OK;
}

#ifndef GW_HOST_FIRST_DIV
#define GW_HOST_FIRST_DIV 8
#endif
static constexpr int64_t kHostFirstDiv = GW_HOST_FIRST_DIV;

gw_status gw_grid_vis_host(gw_plan p, const double* uvw_h, const double* freq_h, int64_t nrow,
                           int32_t nchan, const void* vis_h, const float* weight_h, void* grid,
                           int64_t* n_dropped, void* cuda_stream) {
    gw_status st = common_checks(p, uvw_h, freq_h, nrow, nchan);
    if (st != GW_OK) return st;
    if (!grid) return fail(GW_EINVAL, "null grid");
    if (nrow > 0 && nchan > 0 && !vis_h) return fail(GW_EINVAL, "null vis");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (nrow == 0 || nchan == 0) return finish_dropped(p, n_dropped, s);
    const int npol = p->desc.npol;
    const size_t vb = dtype_bytes(p->desc.vis_dtype);
    // pipeline steps: a short first step (1/kHostFirstDiv of the rows), whose
    // copy is the only one left exposed, then steps of the rest up to the
    // plan's chunk; the second step's copy overlaps the first step's
    // gridding.  Each step beyond one adds a gridding pass (commits, launch
    // tails).  On the 8.26M-visibility batch, with the grid's read-back
    // overlapping the next call: first step 1/2 / 1/4 / 1/8 / 1/16 of the rows
    // 10.2-10.3 / 9.7 / 9.6 / 10.0 ms per call.
    const int64_t rpc = rows_per_chunk(p, nchan);
    const int64_t first = std::max<int64_t>(1, std::min(rpc, (nrow + kHostFirstDiv - 1) / kHostFirstDiv));
    const int64_t rows = std::max<int64_t>(1, std::min(rpc, nrow - first));
    st = ensure_host_pipe(p, std::max(first, rows), nchan);
    if (st != GW_OK) return st;
    e = cudaMemcpyAsync(p->h_freq, freq_h, sizeof(double) * nchan, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copying frequencies");
    // the copy stream may start only after the call's earlier work on s
    e = cudaEventRecord(p->h_free[0], s);
    if (e == cudaSuccess) e = cudaEventRecord(p->h_free[1], s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    int b = 0;
    for (int64_t r0 = 0; r0 < nrow; r0 += (r0 == 0 ? first : rows), b ^= 1) {
        const int64_t nr = std::min(r0 == 0 ? first : rows, nrow - r0);
        const int64_t nv = nr * nchan;
        // copy stream: wait until set b is free, then copy the step's inputs
        e = cudaStreamWaitEvent(p->h_copy, p->h_free[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->h_uvw[b], uvw_h + 3 * r0, sizeof(double) * 3 * nr,
                                cudaMemcpyHostToDevice, p->h_copy);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->h_vis[b], static_cast<const char*>(vis_h) + vb * npol * r0 * nchan,
                                vb * npol * nv, cudaMemcpyHostToDevice, p->h_copy);
        if (e == cudaSuccess && weight_h)
            e = cudaMemcpyAsync(p->h_wt[b], weight_h + (size_t)npol * r0 * nchan,
                                sizeof(float) * npol * nv, cudaMemcpyHostToDevice, p->h_copy);
        if (e == cudaSuccess) e = cudaEventRecord(p->h_ready[b], p->h_copy);
        // compute stream: wait for the copies, grid the step, release set b
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->h_ready[b], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host pipeline copy");
        st = grid_impl(p, p->h_uvw[b], p->h_freq, nr, nchan, p->h_vis[b],
                       weight_h ? p->h_wt[b] : nullptr, grid, nullptr, nullptr, s, false);
        if (st != GW_OK) return st;
        e = cudaEventRecord(p->h_free[b], s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    // the next call's copies must not overtake this call's last gridding
    e = cudaStreamWaitEvent(p->h_copy, p->h_free[b ^ 1], 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    return finish_dropped(p, n_dropped, s);
}

gw_status gw_grid_vis_compensated(gw_plan p, const double* uvw_m, const double* freq_hz,
                                  int64_t nrow, int32_t nchan, const void* vis,
                                  const float* weight, void* grid, void* grid_err,
                                  int64_t* n_dropped, void* cuda_stream) {
    if (!grid_err) return fail(GW_EINVAL, "null grid_err");
    return grid_impl(p, uvw_m, freq_hz, nrow, nchan, vis, weight, grid, grid_err, n_dropped,
                     cuda_stream);
}

static gw_status ensure_compress(gw_plan p, cudaStream_t s) {
    CompressScratch& cs = p->cs;
    if (cs.keys) return GW_OK;
    int64_t cap = 1;
    while (cap < 2 * p->chunk) cap <<= 1;
    const int npol = p->desc.npol;
    cudaError_t e = cudaSuccess;
#define GW_CALLOC(x, n) do { e = dmalloc(&(x), (n)); if (e != cudaSuccess) { \
        dev_free(cs.keys); dev_free(cs.acc); dev_free(cs.rec); dev_free(cs.vis); \
        dev_free(cs.count); cs = CompressScratch{}; \
        return fail(GW_ENOMEM, "allocating compression scratch (%s)", #x); } } while (0)
    GW_CALLOC(cs.keys, (size_t)cap);
    GW_CALLOC(cs.acc, (size_t)cap * npol);
    GW_CALLOC(cs.rec, (size_t)p->chunk);
    GW_CALLOC(cs.vis, (size_t)p->chunk * npol);
    GW_CALLOC(cs.count, 3);
#undef GW_CALLOC
    cs.total = cs.count + 1;
    cs.n_in = cs.count + 2;
    cs.cap = cap;
    clear_compress_table(cs, npol, s);
    return GW_OK;
}

gw_status gw_grid_vis_compressed(gw_plan p, const double* uvw_m, const double* freq_hz,
                                 int64_t nrow, int32_t nchan, const void* vis,
                                 const float* weight, void* grid, int64_t* n_gridded,
                                 int64_t* n_dropped, void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (!grid) return fail(GW_EINVAL, "null grid");
    if (nrow > 0 && nchan > 0 && !vis) return fail(GW_EINVAL, "null vis");
    const int vk = p->desc.vis_dtype;
    const size_t vb = dtype_bytes(vk);
    if ((reinterpret_cast<uintptr_t>(grid) % 8 != 0) || (reinterpret_cast<uintptr_t>(vis) % vb != 0))
        return fail(GW_EINVAL, "grid must be 8-byte aligned and vis aligned to its element size");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    st = ensure_compress(p, s);
    if (st != GW_OK) return st;
    cudaError_t e;
    const int npol = p->desc.npol;
    const int64_t rpc = rows_per_chunk(p, nchan);
    if (p->tuning.compress_min_gain > 0 && nrow > 0 && nchan > 0) {
        // compress a sample (the first rows, up to 2^18 visibilities) and
        // grid without compression when too few of its records merge
        const int64_t sr = std::min(rpc, std::max<int64_t>(1, ((int64_t)1 << 18) / nchan));
        const int64_t nsr = std::min(sr, nrow);
        e = cudaMemsetAsync(p->cs.count, 0, 3 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        launch_index(uvw_m, freq_hz, nsr, nchan, p->ip, p->sc.rec, p->sc.dropped, s);
        launch_compress(p->sc.rec, nsr * nchan, vis, vk, weight, npol, p->desc.oversample, p->cs,
                        s);
        unsigned long long h[3] = {0, 0, 0};
        e = cudaMemcpyAsync(h, p->cs.count, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading the compression sample");
        const double merged = h[2] ? 1.0 - (double)h[0] / (double)h[2] : 0.0;
        if (merged * 1000.0 < (double)p->tuning.compress_min_gain) {
            int64_t nd = 0;
            st = grid_impl(p, uvw_m, freq_hz, nrow, nchan, vis, weight, grid, nullptr, &nd,
                           cuda_stream);
            if (st != GW_OK) return st;
            if (n_dropped) *n_dropped = nd;
            if (n_gridded) *n_gridded = nrow * (int64_t)nchan - nd;
            return GW_OK;
        }
    }
    e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->cs.total, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    for (int64_t r0 = 0; r0 < nrow && nchan > 0; r0 += rpc) {
        const int64_t nr = std::min(rpc, nrow - r0);
        const int64_t v0 = r0 * nchan;
        const int64_t nv = nr * nchan;
        {
            StageTimer t(p, kStIndex, s);
            launch_index(uvw_m + 3 * r0, freq_hz, nr, nchan, p->ip, p->sc.rec, p->sc.dropped, s);
        }
        launch_compress(p->sc.rec, nv, static_cast<const char*>(vis) + (size_t)v0 * npol * vb, vk,
                        weight ? weight + v0 * npol : nullptr, npol, p->desc.oversample, p->cs, s);
        // bin and grid the compressed records (count read on the device)
        const DevCount dc{reinterpret_cast<const int64_t*>(p->cs.count), 1};
        {
            StageTimer t(p, kStBin, s);
            launch_bin(p->cs.rec, nv, p->geom_grid, p->desc.n_wplanes, p->desc.support_min,
                       p->desc.support_max, p->sc, s, dc);
        }
        GridArgs a;
        a.rec = p->cs.rec;
        a.ptable = p->ptable;
        a.pplane_off = p->d_pplane_off;
        a.vis = p->cs.vis;
        a.vis_kind = GW_C64;
        a.weight = nullptr;
        a.table_kind = p->grid_tk;
        a.table_inv = p->table_inv;
        a.plane_off = p->d_plane_off;
        a.support = p->d_support;
        a.entries = p->sc.entries;
        a.items = p->sc.items;
        a.item_count = p->sc.item_off + p->geom_grid.ntu * p->geom_grid.ntv;
        a.queue = p->sc.counters;
        a.grid = reinterpret_cast<float2*>(grid);
        a.grid_err = nullptr;
        a.N = p->desc.grid_n;
        a.npol = npol;
        a.beta = p->desc.oversample;
        a.ntiles_u = p->geom_grid.ntu;
        a.pad_stride = p->pad_stride;
        a.ptable_elems = p->pplane_off.back();
        {
            StageTimer t(p, kStGrid, s);
            launch_grid(a, p->num_sms, s);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "compressed grid launch");
    }
    if (n_gridded) {
        unsigned long long h = 0;
        e = cudaMemcpyAsync(&h, p->cs.total, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading the compressed count");
        *n_gridded = (int64_t)h;
    }
    return finish_dropped(p, n_dropped, s);
}

static gw_status ensure_wstack(gw_plan p, int nlayers) {
    if (p->ws_layers >= nlayers) return GW_OK;
    dev_free(p->ws_count);
    dev_free(p->ws_offsets);
    dev_free(p->ws_cursor);
    dev_free(p->ws_item_off);
    dev_free(p->ws_items);
    p->ws_count = p->ws_offsets = p->ws_cursor = p->ws_item_off = nullptr;
    p->ws_items = nullptr;
    p->ws_layers = 0;
    const int64_t nt = (int64_t)nlayers * p->geom_grid.ntu * p->geom_grid.ntv;
    if (nt >= ((int64_t)1 << 31)) return fail(GW_EINVAL, "too many layer tiles");
    const int64_t icap = p->sc.entries_cap / kItemMin + nt + 1;
    cudaError_t e = dmalloc(&p->ws_count, (size_t)nt);
    if (e == cudaSuccess) e = dmalloc(&p->ws_offsets, (size_t)nt + 1);
    if (e == cudaSuccess) e = dmalloc(&p->ws_cursor, (size_t)nt);
    if (e == cudaSuccess) e = dmalloc(&p->ws_item_off, (size_t)nt + 1);
    if (e == cudaSuccess) e = dmalloc(&p->ws_items, (size_t)icap);
    if (e != cudaSuccess) {
        dev_free(p->ws_count);
        dev_free(p->ws_offsets);
        dev_free(p->ws_cursor);
        dev_free(p->ws_item_off);
        dev_free(p->ws_items);
        p->ws_count = p->ws_offsets = p->ws_cursor = p->ws_item_off = nullptr;
        p->ws_items = nullptr;
        return fail(GW_ENOMEM, "allocating w-stacking bins");
    }
    p->ws_layers = nlayers;
    p->ws_items_cap = icap;
    return GW_OK;
}

gw_status gw_grid_vis_wstack(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                             int32_t nchan, const void* vis, const float* weight,
                             int32_t n_layers, double w_min_lambda, double w_max_lambda,
                             void* layers, int64_t* n_dropped, void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (p->desc.n_wplanes != 1)
        return fail(GW_EINVAL, "w-stacking needs a 2-D plan (n_wplanes == 1)");
    if (n_layers < 1 || n_layers > 4096) return fail(GW_EINVAL, "n_layers must be in [1, 4096]");
    if (!std::isfinite(w_min_lambda) || !std::isfinite(w_max_lambda) ||
        (n_layers > 1 && !(w_max_lambda > w_min_lambda)))
        return fail(GW_EINVAL, "w range must be finite with w_max > w_min");
    if (!layers) return fail(GW_EINVAL, "null layers");
    if (nrow > 0 && nchan > 0 && !vis) return fail(GW_EINVAL, "null vis");
    const int vk = p->desc.vis_dtype;
    const size_t vb = dtype_bytes(vk);
    if ((reinterpret_cast<uintptr_t>(layers) % 8 != 0) ||
        (reinterpret_cast<uintptr_t>(vis) % vb != 0))
        return fail(GW_EINVAL, "layers must be 8-byte aligned and vis aligned to its element size");
    st = ensure_wstack(p, n_layers);
    if (st != GW_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    IndexParams ip = p->ip;
    ip.nlayers = n_layers;
    ip.wmin = w_min_lambda;
    ip.dw = n_layers > 1 ? (w_max_lambda - w_min_lambda) / (double)(n_layers - 1) : 1.0;
    BinGeom g = p->geom_grid;
    g.layer_tiles = g.ntu * g.ntv;
    g.nlayers = n_layers;
    Scratch sc = p->sc;
    sc.count = p->ws_count;
    sc.offsets = p->ws_offsets;
    sc.cursor = p->ws_cursor;
    sc.item_off = p->ws_item_off;
    sc.items = p->ws_items;
    sc.items_cap = p->ws_items_cap;
    const int npol = p->desc.npol;
    const int64_t rpc = rows_per_chunk(p, nchan);
    for (int64_t r0 = 0; r0 < nrow && nchan > 0; r0 += rpc) {
        const int64_t nr = std::min(rpc, nrow - r0);
        const int64_t v0 = r0 * nchan;
        {
            StageTimer t(p, kStIndex, s);
            launch_index(uvw_m + 3 * r0, freq_hz, nr, nchan, ip, sc.rec, sc.dropped, s);
        }
        {
            StageTimer t(p, kStBin, s);
            launch_bin(sc.rec, nr * (int64_t)nchan, g, 1, p->desc.support_min,
                       p->desc.support_min, sc, s);
        }
        GridArgs a;
        a.rec = sc.rec;
        a.ptable = p->ptable;
        a.pplane_off = p->d_pplane_off;
        a.vis = static_cast<const char*>(vis) + (size_t)v0 * npol * vb;
        a.vis_kind = vk;
        a.weight = weight ? weight + v0 * npol : nullptr;
        a.table_kind = p->grid_tk;
        a.table_inv = p->table_inv;
        a.plane_off = p->d_plane_off;
        a.support = p->d_support;
        a.entries = sc.entries;
        a.items = sc.items;
        a.item_count = sc.item_off + (int64_t)g.layer_tiles * n_layers;
        a.queue = sc.counters;
        a.grid = reinterpret_cast<float2*>(layers);
        a.grid_err = nullptr;
        a.N = p->desc.grid_n;
        a.npol = npol;
        a.beta = p->desc.oversample;
        a.ntiles_u = g.ntu;
        a.pad_stride = p->pad_stride;
        a.ptable_elems = p->pplane_off.back();
        a.layer_tiles = g.layer_tiles;
        a.layer_stride = (int64_t)npol * p->desc.grid_n * p->desc.grid_n;
        {
            StageTimer t(p, kStGrid, s);
            launch_grid(a, p->num_sms, s);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "w-stacking grid launch");
    }
    return finish_dropped(p, n_dropped, s);
}

gw_status gw_wstack_combine(gw_plan p, const void* layer_images, int32_t n_layers,
                            double w_min_lambda, double w_max_lambda, void* image,
                            void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    if (!layer_images || !image) return fail(GW_EINVAL, "null argument");
    if (n_layers < 1 || n_layers > 4096) return fail(GW_EINVAL, "n_layers must be in [1, 4096]");
    const double dw = n_layers > 1 ? (w_max_lambda - w_min_lambda) / (double)(n_layers - 1) : 1.0;
    launch_wstack_combine(reinterpret_cast<const float2*>(layer_images), n_layers, w_min_lambda, dw,
                          p->desc.grid_n, p->desc.npol, p->desc.cell_rad,
                          reinterpret_cast<float2*>(image), (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "w-stacking combine launch");
}

static gw_status hybrid_checks(gw_plan p, int32_t sz) {
    if (p->desc.n_wplanes != 1) return fail(GW_EINVAL, "hybrid gridding needs a 2-D plan");
    if (sz < 1 || !(sz & 1) || sz > 127) return fail(GW_EINVAL, "sz must be odd in [1, 127]");
    if (p->desc.grid_n % 4 != 0) return fail(GW_EINVAL, "hybrid gridding needs grid_n %% 4 == 0");
    if (p->desc.oversample % 4 != 0)
        return fail(GW_EINVAL, "hybrid gridding needs oversample %% 4 == 0");
    if ((int64_t)p->desc.oversample * p->desc.grid_n >= ((int64_t)1 << 31))
        return fail(GW_EINVAL, "oversample * grid_n too large");
    return GW_OK;
}

static gw_status ensure_prune(gw_plan p, int32_t sz, cudaStream_t s) {
    if (p->hy_sz == sz) return GW_OK;
    dev_free(p->d_z);
    dev_free(p->d_hpr);
    dev_free(p->d_hprf);
    p->d_z = nullptr;
    p->d_hpr = nullptr;
    p->d_hprf = nullptr;
    p->hy_sz = 0;
    const int N = p->desc.grid_n, beta = p->desc.oversample;
    cudaError_t e = dmalloc(&p->d_z, (size_t)(beta / 2) * sz);
    if (e == cudaSuccess) e = dmalloc(&p->d_hpr, (size_t)N);
    if (e == cudaSuccess) e = dmalloc(&p->d_hprf, (size_t)N);
    if (e != cudaSuccess) {
        dev_free(p->d_z);
        dev_free(p->d_hpr);
        dev_free(p->d_hprf);
        p->d_z = nullptr;
        p->d_hpr = nullptr;
        p->d_hprf = nullptr;
        return fail(GW_ENOMEM, "allocating the pruner");
    }
    e = build_prune(sz, beta, N, p->d_z, p->d_hpr, p->d_hprf, s);
    if (e != cudaSuccess) return cuda_fail(e, "building the pruner");
    p->h_z.assign((size_t)(beta / 2) * sz, 0.f);
    e = cudaMemcpyAsync(p->h_z.data(), p->d_z, sizeof(float) * p->h_z.size(),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "copying the pruning table");
    p->hy_sz = sz;
    return GW_OK;
}

gw_status gw_hybrid_grid(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                         int32_t nchan, const void* vis, const float* weight, int32_t sz,
                         void* fine, int64_t* n_dropped, void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    st = hybrid_checks(p, sz);
    if (st != GW_OK) return st;
    if (!fine) return fail(GW_EINVAL, "null fine grid");
    if (nrow > 0 && nchan > 0 && !vis) return fail(GW_EINVAL, "null vis");
    const int vk = p->desc.vis_dtype;
    const size_t vb = dtype_bytes(vk);
    const uintptr_t fa = (p->desc.npol % 2 == 0) ? 16 : 8;     // vector atomics over pol pairs
    if ((reinterpret_cast<uintptr_t>(fine) % fa != 0) || (reinterpret_cast<uintptr_t>(vis) % vb != 0))
        return fail(GW_EINVAL, "fine must be 16-byte aligned (8 for odd npol) and vis aligned to "
                               "its element size");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const int npol = p->desc.npol;
    const int64_t rpc = rows_per_chunk(p, nchan);
    for (int64_t r0 = 0; r0 < nrow && nchan > 0; r0 += rpc) {
        const int64_t nr = std::min(rpc, nrow - r0);
        const int64_t v0 = r0 * nchan;
        {
            StageTimer t(p, kStIndex, s);
            launch_index(uvw_m + 3 * r0, freq_hz, nr, nchan, p->ip, p->sc.rec, p->sc.dropped, s);
        }
        {
            StageTimer t(p, kStGrid, s);
            launch_hybrid_grid(p->sc.rec, nr * nchan, static_cast<const char*>(vis) + v0 * npol * vb,
                               vk, weight ? weight + v0 * npol : nullptr, npol,
                               p->desc.oversample, p->support[0], p->d_c1, p->c1_fmin,
                               p->c1_norm, p->desc.grid_n, sz, reinterpret_cast<float2*>(fine),
                               p->sc.dropped, s);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "hybrid grid launch");
    }
    return finish_dropped(p, n_dropped, s);
}

gw_status gw_hybrid_prune(gw_plan p, int32_t sz, const void* fine, void* pruned,
                          void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    st = hybrid_checks(p, sz);
    if (st != GW_OK) return st;
    if (!fine || !pruned) return fail(GW_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    st = ensure_prune(p, sz, s);
    if (st != GW_OK) return st;
    launch_prune(reinterpret_cast<const float2*>(fine), p->desc.npol, p->desc.grid_n,
                 p->desc.oversample, sz, p->d_z, p->h_z.data(), p->num_sms,
                 reinterpret_cast<float2*>(pruned), s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "prune launch");
}

gw_status gw_hybrid_shift(gw_plan p, void* pruned, void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    if (!pruned) return fail(GW_EINVAL, "null argument");
    launch_hybrid_shift(reinterpret_cast<float2*>(pruned), p->desc.npol, p->desc.grid_n,
                        (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "hybrid shift launch");
}

gw_status gw_hybrid_image(gw_plan p, int32_t sz, const void* raw, void* image, void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    st = hybrid_checks(p, sz);
    if (st != GW_OK) return st;
    if (!raw || !image) return fail(GW_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    st = ensure_prune(p, sz, s);
    if (st != GW_OK) return st;
    launch_hybrid_image(reinterpret_cast<const float2*>(raw), p->desc.npol, p->desc.grid_n,
                        p->d_hf, p->d_hprf, reinterpret_cast<float2*>(image), s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "hybrid image launch");
}

gw_status gw_grid_fold(gw_plan p, void* grid, void* grid_err, void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    if (!grid || !grid_err) return fail(GW_EINVAL, "null grid or grid_err");
    const int64_t n = (int64_t)p->desc.npol * p->desc.grid_n * p->desc.grid_n;
    launch_fold(reinterpret_cast<float2*>(grid), reinterpret_cast<float2*>(grid_err), n,
                (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "fold launch");
}

gw_status gw_degrid_vis(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                        int32_t nchan, const void* grid, void* vis_out, int64_t* n_dropped,
                        void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (!grid) return fail(GW_EINVAL, "null grid");
    if (nrow > 0 && nchan > 0 && !vis_out) return fail(GW_EINVAL, "null vis_out");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const int npol = p->desc.npol;
    const size_t vb = dtype_bytes(p->desc.vis_dtype);
    if (reinterpret_cast<uintptr_t>(vis_out) % vb != 0)
        return fail(GW_EINVAL, "vis_out must be aligned to its element size");
    const int64_t rpc = rows_per_chunk(p, nchan);
    for (int64_t r0 = 0; r0 < nrow && nchan > 0; r0 += rpc) {
        const int64_t nr = std::min(rpc, nrow - r0);
        const int64_t v0 = r0 * nchan;
        void* out = static_cast<char*>(vis_out) + (size_t)v0 * npol * vb;
        e = cudaMemsetAsync(out, 0, vb * nr * nchan * npol, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        const bool staged = p->tuning.degrid_kernel != 2 && degrid_staged_fits(p->hmax, npol);
        const BinGeom& geom = staged ? p->geom_staged : p->geom_degrid;
        st = index_and_bin(p, uvw_m + 3 * r0, freq_hz, nr, nchan, geom, s);
        if (st != GW_OK) return st;
        DegridArgs a;
        a.rec = p->sc.rec;
        a.grid = reinterpret_cast<const float2*>(grid);
        a.table = p->table16 ? (const void*)p->table16 : (const void*)p->table;
        a.table_kind = p->desc.table_dtype;
        a.vis_kind = p->desc.vis_dtype;
        a.table_inv = p->table_inv;
        a.table_elems = p->plane_off.back() + kTableSlack;
        a.plane_off = p->d_plane_off;
        a.support = p->d_support;
        a.entries = p->sc.entries;
        a.n_entries = p->sc.offsets + geom.ntu * geom.ntv;
        a.vis_out = out;
        a.vis_count = nr * (int64_t)nchan;
        a.N = p->desc.grid_n;
        a.npol = npol;
        a.beta = p->desc.oversample;
        a.items = p->sc.items;
        a.item_count = p->sc.item_off + geom.ntu * geom.ntv;
        a.queue = p->sc.counters;
        a.ntiles_u = geom.ntu;
        {
            StageTimer t(p, kStDegrid, s);
            if (!(staged && launch_degrid_staged(a, p->hmax, p->num_sms, s)))
                launch_degrid(a, nr * nchan, p->num_sms, s);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "degrid launch");
    }
    return finish_dropped(p, n_dropped, s);
}

// Shared checks of the device-count entry points; the whole call is one chunk.
static gw_status devcount_checks(gw_plan p, const double* uvw_m, const double* freq_hz,
                                 const int64_t* d_nrow, int64_t max_nrow, int32_t nchan,
                                 const void* a, const void* b) {
    gw_status st = common_checks(p, uvw_m, freq_hz, max_nrow, nchan);
    if (st != GW_OK) return st;
    if (!d_nrow || !a || !b) return fail(GW_EINVAL, "null argument");
    if (max_nrow * (int64_t)nchan > p->chunk)
        return fail(GW_EINVAL, "max_nrow * nchan (%lld) exceeds the plan's chunk (%lld): "
                    "clone the plan with a larger max_vis_per_call",
                    (long long)(max_nrow * (int64_t)nchan), (long long)p->chunk);
    return GW_OK;
}

gw_status gw_grid_vis_devcount(gw_plan p, const double* uvw_m, const double* freq_hz,
                               const int64_t* d_nrow, int64_t max_nrow, int32_t nchan,
                               const void* vis, void* grid, void* cuda_stream) {
    gw_status st = devcount_checks(p, uvw_m, freq_hz, d_nrow, max_nrow, nchan, vis, grid);
    if (st != GW_OK) return st;
    const int vk = p->desc.vis_dtype;
    if ((reinterpret_cast<uintptr_t>(grid) % 8 != 0) ||
        (reinterpret_cast<uintptr_t>(vis) % dtype_bytes(vk) != 0))
        return fail(GW_EINVAL, "grid must be 8-byte aligned and vis aligned to its element size");
    if (max_nrow == 0 || nchan == 0) return GW_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const DevCount dc{d_nrow, nchan};
    launch_index(uvw_m, freq_hz, max_nrow, nchan, p->ip, p->sc.rec, p->sc.dropped, s, d_nrow);
    launch_bin(p->sc.rec, max_nrow * (int64_t)nchan, p->geom_grid, p->desc.n_wplanes,
               p->desc.support_min, p->desc.support_max, p->sc, s, dc);
    GridArgs a;
    a.rec = p->sc.rec;
    a.ptable = p->ptable;
    a.pplane_off = p->d_pplane_off;
    a.vis = vis;
    a.vis_kind = vk;
    a.weight = nullptr;
    a.table_kind = p->grid_tk;
    a.table_inv = p->table_inv;
    a.plane_off = p->d_plane_off;
    a.support = p->d_support;
    a.entries = p->sc.entries;
    a.items = p->sc.items;
    a.item_count = p->sc.item_off + p->geom_grid.ntu * p->geom_grid.ntv;
    a.queue = p->sc.counters;
    a.grid = reinterpret_cast<float2*>(grid);
    a.grid_err = nullptr;
    a.N = p->desc.grid_n;
    a.npol = p->desc.npol;
    a.beta = p->desc.oversample;
    a.ntiles_u = p->geom_grid.ntu;
    a.pad_stride = p->pad_stride;
    a.ptable_elems = p->pplane_off.back();
    launch_grid(a, p->num_sms, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "grid launch");
}

gw_status gw_grid_vis_devcount_readback(gw_plan p, const double* uvw_m, const double* freq_hz,
                                        const int64_t* d_nrow, int64_t max_nrow, int32_t nchan,
                                        const void* vis, void* grid, void* host_grid,
                                        int32_t n_bands, void* cuda_stream) {
    gw_status st = devcount_checks(p, uvw_m, freq_hz, d_nrow, max_nrow, nchan, vis, grid);
    if (st != GW_OK) return st;
    if (!host_grid) return fail(GW_EINVAL, "null host_grid");
    if (n_bands < 1 || n_bands > kReadbackBandsMax)
        return fail(GW_EINVAL, "n_bands must be in [1, %d]", kReadbackBandsMax);
    const int vk = p->desc.vis_dtype;
    if ((reinterpret_cast<uintptr_t>(grid) % 8 != 0) ||
        (reinterpret_cast<uintptr_t>(host_grid) % 8 != 0) ||
        (reinterpret_cast<uintptr_t>(vis) % dtype_bytes(vk) != 0))
        return fail(GW_EINVAL, "grid and host_grid must be 8-byte aligned and vis aligned to its "
                    "element size");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    // copy stream and events (outside any capture: the first call creates them)
    if (!p->rb_stream) {
        e = cudaStreamCreateWithFlags(&p->rb_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            p->rb_stream = nullptr;
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
    }
    while ((int)p->rb_ev.size() < n_bands + 1) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        p->rb_ev.push_back(ev);
    }
    const int N = p->desc.grid_n, npol = p->desc.npol;
    const int ntu = p->geom_grid.ntu, ntv = p->geom_grid.ntv;
    const int nb = std::min(n_bands, ntv);
    float2* g = reinterpret_cast<float2*>(grid);
    float2* h = reinterpret_cast<float2*>(host_grid);
    auto copy_rows = [&](int r0, int r1) -> cudaError_t {
        cudaError_t ce = cudaSuccess;
        for (int q = 0; q < npol && ce == cudaSuccess && r1 > r0; ++q) {
            const size_t off = ((size_t)q * N + r0) * N;
            ce = cudaMemcpyAsync(h + off, g + off, sizeof(float2) * (size_t)(r1 - r0) * N,
                                 cudaMemcpyDeviceToHost, p->rb_stream);
        }
        return ce;
    };
    if (max_nrow > 0 && nchan > 0) {
        e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        const DevCount dc{d_nrow, nchan};
        launch_index(uvw_m, freq_hz, max_nrow, nchan, p->ip, p->sc.rec, p->sc.dropped, s, d_nrow);
        launch_bin(p->sc.rec, max_nrow * (int64_t)nchan, p->geom_grid, p->desc.n_wplanes,
                   p->desc.support_min, p->desc.support_max, p->sc, s, dc);
    }
    GridArgs a;
    a.rec = p->sc.rec;
    a.ptable = p->ptable;
    a.pplane_off = p->d_pplane_off;
    a.vis = vis;
    a.vis_kind = vk;
    a.weight = nullptr;
    a.table_kind = p->grid_tk;
    a.table_inv = p->table_inv;
    a.plane_off = p->d_plane_off;
    a.support = p->d_support;
    a.entries = p->sc.entries;
    a.items = p->sc.items;
    a.queue = p->sc.counters;
    a.grid = g;
    a.grid_err = nullptr;
    a.N = N;
    a.npol = npol;
    a.beta = p->desc.oversample;
    a.ntiles_u = ntu;
    a.pad_stride = p->pad_stride;
    a.ptable_elems = p->pplane_off.back();
    // band b: tile rows [b ntv / nb, (b + 1) ntv / nb), its work items the
    // contiguous run item_off[first tile] .. item_off[first tile of the next
    // band]; its grid rows are final once its launch ends (no other band's
    // items touch its tiles), so they are copied while the next band grids
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        const int tv0 = (int)((int64_t)b * ntv / nb), tv1 = (int)((int64_t)(b + 1) * ntv / nb);
        if (max_nrow > 0 && nchan > 0) {
            a.item_first = p->sc.item_off + tv0 * ntu;
            a.item_count = p->sc.item_off + tv1 * ntu;
            launch_grid(a, p->num_sms, s);
        }
        e = cudaEventRecord(p->rb_ev[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->rb_stream, p->rb_ev[b], 0);
        if (e == cudaSuccess)
            e = copy_rows(tv0 * kGridTileV, std::min(tv1 * kGridTileV, N));
    }
    // the caller's stream continues after the last copy
    if (e == cudaSuccess) e = cudaEventRecord(p->rb_ev[nb], p->rb_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->rb_ev[nb], 0);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "banded gridding and read-back");
}

gw_status gw_degrid_vis_devcount(gw_plan p, const double* uvw_m, const double* freq_hz,
                                 const int64_t* d_nrow, int64_t max_nrow, int32_t nchan,
                                 const void* grid, void* vis_out, void* cuda_stream) {
    gw_status st = devcount_checks(p, uvw_m, freq_hz, d_nrow, max_nrow, nchan, grid, vis_out);
    if (st != GW_OK) return st;
    const int vk = p->desc.vis_dtype, npol = p->desc.npol;
    if (reinterpret_cast<uintptr_t>(vis_out) % dtype_bytes(vk) != 0)
        return fail(GW_EINVAL, "vis_out must be aligned to its element size");
    if (max_nrow == 0 || nchan == 0) return GW_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const DevCount dc{d_nrow, nchan};
    const int64_t nmax = max_nrow * (int64_t)nchan;
    launch_zero_vis(vis_out, vk, nmax, npol, dc, s);
    const bool staged = p->tuning.degrid_kernel != 2 && degrid_staged_fits(p->hmax, npol);
    const BinGeom& geom = staged ? p->geom_staged : p->geom_degrid;
    launch_index(uvw_m, freq_hz, max_nrow, nchan, p->ip, p->sc.rec, p->sc.dropped, s, d_nrow);
    launch_bin(p->sc.rec, nmax, geom, p->desc.n_wplanes, p->desc.support_min,
               p->desc.support_max, p->sc, s, dc);
    DegridArgs a;
    a.rec = p->sc.rec;
    a.grid = reinterpret_cast<const float2*>(grid);
    a.table = p->table16 ? (const void*)p->table16 : (const void*)p->table;
    a.table_kind = p->desc.table_dtype;
    a.vis_kind = vk;
    a.table_inv = p->table_inv;
    a.table_elems = p->plane_off.back() + kTableSlack;
    a.plane_off = p->d_plane_off;
    a.support = p->d_support;
    a.entries = p->sc.entries;
    a.n_entries = p->sc.offsets + geom.ntu * geom.ntv;
    a.vis_out = vis_out;
    a.vis_count = max_nrow * (int64_t)nchan;
    a.N = p->desc.grid_n;
    a.npol = npol;
    a.beta = p->desc.oversample;
    a.items = p->sc.items;
    a.item_count = p->sc.item_off + geom.ntu * geom.ntv;
    a.queue = p->sc.counters;
    a.ntiles_u = geom.ntu;
    if (!(staged && launch_degrid_staged(a, p->hmax, p->num_sms, s)))
        launch_degrid(a, nmax, p->num_sms, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "degrid launch");
}

gw_status gw_degrid_vis_static(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                               int32_t nchan, const void* grid, void* vis_out, int64_t* n_dropped,
                               void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (!grid) return fail(GW_EINVAL, "null grid");
    if (nrow > 0 && nchan > 0 && !vis_out) return fail(GW_EINVAL, "null vis_out");
    const int64_t nvis = nrow * (int64_t)nchan;
    if (reinterpret_cast<uintptr_t>(vis_out) % dtype_bytes(p->desc.vis_dtype) != 0)
        return fail(GW_EINVAL, "vis_out must be aligned to its element size");
    if (nvis > static_scratch_max_vis())
        return fail(GW_EINVAL, "gw_degrid_vis_static: %lld visibilities exceed the static scratch "
                    "limit of %lld per call", (long long)nvis, (long long)static_scratch_max_vis());
    const BinGeom& g = p->geom_degrid;
    if (g.ntu * g.ntv > static_scratch_max_tiles())
        return fail(GW_EINVAL, "gw_degrid_vis_static: grid_n %d needs %d tiles, the static scratch "
                    "holds %d (grid_n <= 8192)", p->desc.grid_n, g.ntu * g.ntv,
                    static_scratch_max_tiles());
    Scratch sc;
    cudaError_t e = static_scratch_view(&sc);
    if (e != cudaSuccess) return cuda_fail(e, "locating the static scratch (cudaGetSymbolAddress)");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: reset what must start at zero
    e = cudaMemsetAsync(sc.dropped, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.work, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && nvis > 0)
        e = cudaMemsetAsync(vis_out, 0, (size_t)dtype_bytes(p->desc.vis_dtype) * nvis * p->desc.npol, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (nvis > 0) {
        launch_index(uvw_m, freq_hz, nrow, nchan, p->ip, sc.rec, sc.dropped, s);
        launch_bin(sc.rec, nvis, g, p->desc.n_wplanes, p->desc.support_min, p->desc.support_max,
                   sc, s);
        DegridArgs a;
        a.rec = sc.rec;
        a.grid = reinterpret_cast<const float2*>(grid);
        a.table = p->table16 ? (const void*)p->table16 : (const void*)p->table;
        a.table_kind = p->desc.table_dtype;
        a.vis_kind = p->desc.vis_dtype;
        a.table_inv = p->table_inv;
        a.table_elems = p->plane_off.back() + kTableSlack;
        a.plane_off = p->d_plane_off;
        a.support = p->d_support;
        a.entries = sc.entries;
        a.n_entries = sc.offsets + g.ntu * g.ntv;
        a.vis_out = vis_out;
        a.vis_count = nrow * (int64_t)nchan;
        a.N = p->desc.grid_n;
        a.npol = p->desc.npol;
        a.beta = p->desc.oversample;
        launch_degrid(a, nvis, p->num_sms, s);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "static degrid launch");
    }
    if (!n_dropped) return GW_OK;
    unsigned long long h = 0;
    e = cudaMemcpyAsync(&h, sc.dropped, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the drop count");
    *n_dropped = (int64_t)h;
    return GW_OK;
}

gw_status gw_grid_correct(gw_plan p, void* image, int32_t direction, void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    if (!image) return fail(GW_EINVAL, "null image");
    if (direction < -1 || direction > 1) return fail(GW_EINVAL, "direction must be -1, 0 or +1");
    launch_correct(reinterpret_cast<float2*>(image), p->d_hf, p->desc.grid_n, p->desc.npol,
                   direction, (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "correct launch");
}

gw_status gw_grid_shift(gw_plan p, void* grid, void* cuda_stream) {
    if (!p) return fail(GW_EINVAL, "null plan");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    if (!grid) return fail(GW_EINVAL, "null grid");
    launch_shift(reinterpret_cast<float2*>(grid), p->desc.grid_n, p->desc.npol,
                 (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "shift launch");
}

gw_status gw_index_vis(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                       int32_t nchan, gw_index_rec* out, int64_t* n_dropped, void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (nrow > 0 && nchan > 0 && !out) return fail(GW_EINVAL, "null output");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(p->sc.dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    launch_index(uvw_m, freq_hz, nrow, nchan, p->ip, out, p->sc.dropped, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "index launch");
    return finish_dropped(p, n_dropped, s);
}

gw_status gw_plan_copy_tables(gw_plan p, float* out, int64_t* plane_offsets, int32_t* supports) {
    if (!p || !out) return fail(GW_EINVAL, "null argument");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    cudaError_t e = cudaMemcpy(out, p->table, sizeof(float2) * p->plane_off.back(),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copying tables");
    if (plane_offsets)
        for (size_t i = 0; i < p->plane_off.size(); ++i) plane_offsets[i] = p->plane_off[i];
    if (supports)
        for (size_t i = 0; i < p->support.size(); ++i) supports[i] = p->support[i];
    return GW_OK;
}

gw_status gw_plan_copy_stored_tables(gw_plan p, void* out) {
    if (!p || !out) return fail(GW_EINVAL, "null argument");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    const void* src = p->table16 ? (const void*)p->table16 : (const void*)p->table;
    cudaError_t e = cudaMemcpy(out, src, (size_t)dtype_bytes(p->desc.table_dtype) * p->plane_off.back(),
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "copying stored tables");
}

gw_status gw_ffma_peak(int32_t iters, double* tflops, void* cuda_stream) {
    if (!tflops || iters < 1) return fail(GW_EINVAL, "bad arguments");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = measure_ffma_peak(sms, iters, tflops, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "FFMA probe");
}

gw_status gw_plan_timing_enable(gw_plan p, int32_t enable) {
    if (!p) return fail(GW_EINVAL, "null plan");
    p->timing = enable != 0;
    return GW_OK;
}

gw_status gw_plan_timing_get(gw_plan p, gw_timing* out) {
    if (!p || !out) return fail(GW_EINVAL, "null argument");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    std::memset(out, 0, sizeof *out);
    double* ms[4] = {&out->index_ms, &out->bin_ms, &out->grid_ms, &out->degrid_ms};
    int64_t* calls[4] = {&out->index_calls, &out->bin_calls, &out->grid_calls, &out->degrid_calls};
    cudaError_t e = cudaSuccess;
    for (auto& ev : p->events) {
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev.a, ev.b);
        *ms[ev.stage] += t;
        *calls[ev.stage] += 1;
        p->pool.push_back(ev.a);
        p->pool.push_back(ev.b);
    }
    p->events.clear();
    if (e != cudaSuccess) return cuda_fail(e, "reading stage events");
    unsigned long long w[2] = {0, 0};
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(w, p->sc.work, sizeof w, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->sc.work, 0, sizeof w);
    if (e != cudaSuccess) return cuda_fail(e, "reading work counters");
    out->valid_vis = (int64_t)w[0];
    out->taps = (int64_t)w[1];
    return GW_OK;
}

gw_status gw_plan_copy_corrector(gw_plan p, double* out) {
    if (!p || !out) return fail(GW_EINVAL, "null argument");
    gw_status st = check_device(p);
    if (st != GW_OK) return st;
    cudaError_t e = cudaMemcpy(out, p->d_h, sizeof(double) * p->desc.grid_n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GW_OK : cuda_fail(e, "copying corrector");
}

gw_status gw_debug_bins(gw_plan p, const double* uvw_m, const double* freq_hz, int64_t nrow,
                        int32_t nchan, int32_t mode, int64_t* tile_offsets, uint32_t* entries,
                        int64_t capacity, void* cuda_stream) {
    gw_status st = common_checks(p, uvw_m, freq_hz, nrow, nchan);
    if (st != GW_OK) return st;
    if (!tile_offsets || (mode != 0 && mode != 1)) return fail(GW_EINVAL, "bad arguments");
    if (nrow * (int64_t)nchan > p->chunk) return fail(GW_EINVAL, "input exceeds one chunk");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const BinGeom& g = mode == 0 ? p->geom_grid : p->geom_degrid;
    st = index_and_bin(p, uvw_m, freq_hz, nrow, nchan, g, s);
    if (st != GW_OK) return st;
    std::vector<uint32_t> offs(g.ntu * g.ntv + 1);
    cudaError_t e = cudaMemcpyAsync(offs.data(), p->sc.offsets, sizeof(uint32_t) * offs.size(),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "copying bin offsets");
    for (size_t i = 0; i < offs.size(); ++i) tile_offsets[i] = offs[i];
    const int64_t n = offs.back();
    if (n > capacity || (n > 0 && !entries)) return fail(GW_EINVAL, "entries capacity too small");
    if (n > 0) {
        e = cudaMemcpy(entries, p->sc.entries, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copying bin entries");
    }
    return GW_OK;
}

}  // extern "C"
