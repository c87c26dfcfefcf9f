// Allocation-free degridding: gw_degrid_vis_static.
//
// Some callers cannot call cudaMalloc once they are running: a process whose
// device memory is entirely handed to another allocator at start-up (a
// framework's caching pool, a fixed per-process budget), or a loop that must
// not take the driver's allocation lock between iterations.  For them this
// entry point degrids with the same kernels as gw_degrid_vis but takes its
// scratch (index records and centre-tile bins) from one file-scope device
// array, sized once when the library is loaded, instead of from memory the
// plan allocates per chunk.  The plan still supplies the kernel tables; the
// caller still supplies inputs and outputs.
#include "gw_internal.cuh"

#include <mutex>

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

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_dev_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `device` (which must be current).
// Looked up once per device; in host code the symbol name is only a host-side
// stand-in, so kernels must be given this address instead.
cudaError_t static_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev_addr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_dev_addr[device] = static_cast<unsigned char*>(ptr);
    }
    *out = g_dev_addr[device];
    return cudaSuccess;
}

}  // namespace

int64_t static_scratch_max_vis() { return kStaticMaxVis; }
int static_scratch_max_tiles() { return kStaticMaxTiles; }

cudaError_t static_scratch_view(int device, Scratch* sc) {
    unsigned char* base = nullptr;
    cudaError_t e = static_scratch(device, &base);
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
