// Allocation-free degridding: gw_degrid_vis_static.
//
// Some callers cannot call cudaMalloc once they are running: a process whose
// device memory is entirely handed to another allocator at start-up (a
// framework's caching pool, a fixed per-process budget), or a loop that must
// not take the driver's allocation lock between iterations.  For them this
// entry point degrids with the same kernels as gw_degrid_vis but takes its
// scratch (index records and centre-tile bins) from one file-scope device
// array of kStaticBytes (about 2.25 MiB) instead of from memory the plan
// allocates per chunk.  The plan still supplies the kernel tables; the
// caller still supplies inputs and outputs.  The driver allocates the array
// when it loads this file's module; with lazy module loading (the CUDA
// default) that would be the first allocation-free call itself, so plan
// creation loads the module and every kernel the path launches
// (static_path_prepare) while the caller can still allocate.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int64_t kStaticMaxVis = 65536;     // visibilities per call (nrow * nchan)
constexpr int kStaticMaxTiles = 65536;       // centre-mode tiles: N <= 8192 with 32 x 32 tiles

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffRec = 0;
constexpr size_t kOffEntries = kOffRec + align256(sizeof(gw_index_rec) * kStaticMaxVis);
constexpr size_t kOffCount = kOffEntries + align256(sizeof(uint32_t) * kStaticMaxVis);
constexpr size_t kOffCursor = kOffCount + align256(sizeof(uint32_t) * kStaticMaxTiles);
constexpr size_t kOffOffsets = kOffCursor + align256(sizeof(uint32_t) * kStaticMaxTiles);
constexpr size_t kOffItemOff = kOffOffsets + align256(sizeof(uint32_t) * (kStaticMaxTiles + 1));
constexpr size_t kOffDropped = kOffItemOff + align256(sizeof(uint32_t) * (kStaticMaxTiles + 1));
constexpr size_t kOffWork = kOffDropped + align256(sizeof(unsigned long long));
constexpr size_t kStaticBytes = kOffWork + align256(2 * sizeof(unsigned long long));
static_assert(kStaticBytes <= 4u * 1024u * 1024u, "static scratch stays modest (<= 4 MiB)");

// The scratch itself: every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch on the current device.  In host code
// the symbol name is only a host-side stand-in, so kernels must be given this
// address instead.  Looked up on every call: once the module is loaded the
// lookup allocates nothing, and nothing cached can go stale when a context
// is torn down and created again.
cudaError_t static_scratch(unsigned char** out) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(ptr);
    return cudaSuccess;
}

}  // namespace

int64_t static_scratch_max_vis() { return kStaticMaxVis; }
int static_scratch_max_tiles() { return kStaticMaxTiles; }

cudaError_t static_path_prepare(int npol, int table_kind) {
    unsigned char* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e == cudaSuccess) e = preload_index_kernels();
    if (e == cudaSuccess) e = preload_bin_kernels();
    if (e == cudaSuccess) e = preload_degrid_kernel(npol, table_kind);
    return e;
}

cudaError_t static_scratch_view(Scratch* sc) {
    unsigned char* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e != cudaSuccess) return e;
    *sc = Scratch{};
    sc->rec = reinterpret_cast<gw_index_rec*>(base + kOffRec);
    sc->entries = reinterpret_cast<uint32_t*>(base + kOffEntries);
    sc->count = reinterpret_cast<uint32_t*>(base + kOffCount);
    sc->cursor = reinterpret_cast<uint32_t*>(base + kOffCursor);
    sc->offsets = reinterpret_cast<uint32_t*>(base + kOffOffsets);
    sc->item_off = reinterpret_cast<uint32_t*>(base + kOffItemOff);
    sc->dropped = reinterpret_cast<unsigned long long*>(base + kOffDropped);
    sc->work = reinterpret_cast<unsigned long long*>(base + kOffWork);
    sc->entries_cap = kStaticMaxVis;
    return cudaSuccess;
}

}  // namespace gw
