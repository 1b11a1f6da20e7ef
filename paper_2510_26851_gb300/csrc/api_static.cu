// api_static.cu -- jfof_fof_static: the a1-a7 pipeline of jfof_fof with its
// scratch in a fixed device array owned by the library, for callers that must
// not allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not acceptable -- an
// in-situ analysis hook inside a simulation or framework that owns all device
// memory through its own pool, or a latency-critical path that cannot afford
// the implicit device-wide synchronisation cudaMalloc/cudaFree may perform.
// Such a caller still passes its inputs and outputs, but no workspace.
//
// The scratch is one file-scope __device__ array of kStaticScratchBytes on
// every GPU that loads the library, held until the process exits.  Every call
// shares it: two calls whose work overlaps on the GPU (different streams or
// contexts of the same device, or different host threads) race on it and
// must be serialised by the caller.  Each call initialises every part of the
// scratch it reads, so nothing carries over from the previous call.
#include <mutex>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch for each device.  Host code cannot use
// the symbol itself: in host code its name denotes a host-side stand-in.
std::mutex g_static_lock;
void *g_static_addr[64] = {};

// Looks up (once per device, with that device current) the device address of
// the static scratch.
int static_scratch(int device, void **addr) {
    if (device < 0 || device >= 64) return JFOF_EINVAL;
    std::lock_guard<std::mutex> guard(g_static_lock);
    if (!g_static_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return JFOF_ECUDA;
        g_static_addr[device] = p;
    }
    *addr = g_static_addr[device];
    return JFOF_OK;
}

}  // namespace

extern "C" {

int jfof_fof_static(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, int32_t n_axis, uint32_t flags,
                    int32_t min_size, int32_t *label, int32_t *halo_id, int32_t *count, int32_t *halo_start,
                    int32_t *members, int32_t *n_halos) {
    if (!ctx) return JFOF_EINVAL;
    int e = jfof::check_box(N, L, b);
    if (e) return e;
    int32_t n;
    if ((e = jfof::resolve_n(N, L, b, n_axis, &n))) return e;
    size_t need = 0;
    if ((e = jfof_fof_all_bytes(N, n, &need))) return e;
    if (need > kStaticScratchBytes) return JFOF_ENOMEM;  // larger than the fixed scratch
    if (cudaSetDevice(ctx->device) != cudaSuccess) return JFOF_ECUDA;
    void *ws = nullptr;
    if ((e = static_scratch(ctx->device, &ws))) return e;
    return jfof_fof(ctx, pos, N, L, b, n, flags, min_size, ws, kStaticScratchBytes, label, halo_id, count,
                    halo_start, members, n_halos);
}

}  // extern "C"
