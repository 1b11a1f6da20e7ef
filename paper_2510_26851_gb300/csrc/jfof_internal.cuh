// jfof_internal.cuh -- device helpers shared by the sm_103a kernels of the FoF
// hot path (never by the CPU oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jfof.h"

namespace jfof {

// ---------------------------------------------------------------------------
// Launch geometry: grid-stride kernels launch a multiple of the current
// device's SM count (152 on GB300), queried once per device, so every SM gets
// the same number of resident CTAs.
int num_sms();
constexpr int kBrick = 16;                  // cells per brick side
constexpr int kBrickCells = kBrick * kBrick * kBrick;
constexpr int64_t kDefaultLoopBudget = int64_t(1) << 24;

inline int grid_for(int64_t work, int threads, int per_sm = 8) {
    int64_t want = (work + threads - 1) / threads;
    int64_t cap = int64_t(num_sms()) * per_sm;
    if (want < 1) want = 1;
    return int(want < cap ? want : cap);
}

// One thread per work item (no grid-stride loop): blocks are scheduled in
// order, so the items in flight stay a contiguous window -- better locality
// than a persistent grid whose warps drift apart.
inline unsigned grid_full(int64_t work, int threads) {
    int64_t want = (work + threads - 1) / threads;
    return unsigned(want < 1 ? 1 : want);
}

// Context-wide state passed to kernels by value.
struct DevStatus {
    int *status;        // device word: first latched error code
    int64_t loop_budget;
};

__device__ __forceinline__ void latch(const DevStatus &st, int code) {
    atomicCAS(st.status, 0, code);
}

// ---------------------------------------------------------------------------
// Input normalisation (Algorithm 2 "Wrap positions"): x - L*floor(x/L) with
// IEEE divide and single-rounded multiply/subtract, then >= L or < 0 -> 0.
__device__ __forceinline__ float wrap_coord(float x, float L) {
    float q = floorf(__fdiv_rn(x, L));
    float w = __fsub_rn(x, __fmul_rn(L, q));
    if (w >= L) w = 0.0f;
    if (w < 0.0f) w = 0.0f;
    return w;
}

// Cell coordinate floor(x * (n/L)) clamped to [0, n-1]; inv_cell = f32(n/L)
// computed on the host in double.  NaN converts to 0 (cvt.rmi), so the
// result is always a legal cell.
__device__ __forceinline__ int cell_coord(float x, float inv_cell, int n) {
    int c = __float2int_rd(__fmul_rn(x, inv_cell));
    c = c < 0 ? 0 : c;
    c = c > n - 1 ? n - 1 : c;
    return c;
}

// Brick-major cell-table index of cell (ix, iy, iz); nb bricks per axis.
__device__ __forceinline__ uint64_t cell_table_index(int ix, int iy, int iz, int nb) {
    uint64_t brick = uint64_t(ix >> 4) + uint64_t(nb) * (uint64_t(iy >> 4) + uint64_t(nb) * uint64_t(iz >> 4));
    uint32_t local = uint32_t(ix & 15) + 16u * (uint32_t(iy & 15) + 16u * uint32_t(iz & 15));
    return brick * kBrickCells + local;
}

// ---------------------------------------------------------------------------
// The link predicate (Sec. 2 step (iv), Algorithm 2): minimum-image
// difference per axis, then d2 = (dx*dx + dy*dy) + dz*dz, every operation a
// single IEEE binary32 rounding (no FMA contraction).
__device__ __forceinline__ float min_image(float xj, float xi, float L, float hL) {
    float d = __fsub_rn(xj, xi);
    if (d > hL)
        d = __fsub_rn(d, L);
    else if (d < -hL)
        d = __fadd_rn(d, L);
    return d;
}

__device__ __forceinline__ float pair_d2(float4 p, float4 q, float L, float hL) {
    float dx = min_image(q.x, p.x, L, hL);
    float dy = min_image(q.y, p.y, L, hL);
    float dz = min_image(q.z, p.z, L, hL);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------
// Lock-free union-find over int32 parents with parent[x] <= x, so the root of
// every tree is its smallest element (hook larger root under smaller,
// atomicCAS; path halving with plain stores, which only ever write an
// ancestor of a non-root).  Loads may be stale: every value ever stored is an
// ancestor, so finds still terminate (x strictly decreases) and the CAS
// decides.  Each failed CAS strictly lowers max(ra, rb), so the retry loop
// ends; it is still bounded by the context's budget.
__device__ __forceinline__ int uf_find(int *parent, int x) {
    while (true) {
        int p = parent[x];
        if (p == x) return x;
        int gp = parent[p];
        if (gp == p) return p;
        parent[x] = gp;
        x = gp;
    }
}

// Find without writes (used once the forest is frozen).
__device__ __forceinline__ int uf_find_ro(const int *parent, int x) {
    int p = parent[x];
    while (p != x) {
        x = p;
        p = parent[x];
    }
    return x;
}

__device__ __forceinline__ void uf_unite(int *parent, int a, int b, const DevStatus &st) {
    int ra = uf_find(parent, a);
    int rb = uf_find(parent, b);
    for (int64_t it = 0; it < st.loop_budget; ++it) {
        if (ra == rb) return;
        if (ra < rb) {
            int t = ra;
            ra = rb;
            rb = t;
        }
        int old = atomicCAS(&parent[ra], ra, rb);
        if (old == ra) return;
        ra = uf_find(parent, old);
        rb = uf_find(parent, rb);
    }
    latch(st, JFOF_ETIMEOUT);
}

// uf_unite that also returns a member of the merged component (the root it
// hooked under), for callers that cache component representatives.
__device__ __forceinline__ int uf_unite_rep(int *parent, int a, int b, const DevStatus &st) {
    int ra = uf_find(parent, a);
    int rb = uf_find(parent, b);
    for (int64_t it = 0; it < st.loop_budget; ++it) {
        if (ra == rb) return ra;
        if (ra < rb) {
            int t = ra;
            ra = rb;
            rb = t;
        }
        int old = atomicCAS(&parent[ra], ra, rb);
        if (old == ra) return rb;
        ra = uf_find(parent, old);
        rb = uf_find(parent, rb);
    }
    latch(st, JFOF_ETIMEOUT);
    return rb;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of uint32 values produced by a functor
// op(i) for i in [0, n): out[i] = sum_{k<i} op(k), out[n] = total.
// Reduce-then-scan over tiles of 4096 (256 threads x 16), recursing on the
// tile sums.  tmp must hold scan_tmp_words(n) uint32.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_words(int64_t n);

template <class Op>
__global__ void scan_reduce_kernel(Op op, int64_t n, uint32_t *tile_sums) {
    __shared__ uint32_t red[kScanThreads / 32];
    int64_t base = int64_t(blockIdx.x) * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + int64_t(k) * kScanThreads + threadIdx.x;
        if (i < n) s += op(i);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0u;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) tile_sums[blockIdx.x] = v;
    }
}

// Block-level exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *smem_warps, uint32_t *total) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warps[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? smem_warps[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) smem_warps[lane] = w;
    }
    __syncthreads();
    uint32_t warp_prefix = warp > 0 ? smem_warps[warp - 1] : 0u;
    *total = smem_warps[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

template <class Op>
__global__ void scan_down_kernel(Op op, int64_t n, const uint32_t *tile_prefix, uint32_t *out) {
    __shared__ uint32_t warps[kScanThreads / 32];
    int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? op(i) : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t pre = block_exclusive_scan(s, warps, &total) + tile_prefix[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = pre;
        pre += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_prefix[blockIdx.x] + total;
}

struct LoadU32 {
    const uint32_t *p;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return p[i]; }
};

// Exclusive scan of the nt tile sums in place (recursive; host side).
void scan_tiles_inplace(uint32_t *sums, int64_t nt, uint32_t *tmp, cudaStream_t s);

template <class Op>
void scan_exclusive(Op op, int64_t n, uint32_t *out, uint32_t *tmp, cudaStream_t s) {
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt < 1) nt = 1;
    scan_reduce_kernel<Op><<<unsigned(nt), kScanThreads, 0, s>>>(op, n, tmp);
    scan_tiles_inplace(tmp, nt, tmp + nt + 1, s);
    scan_down_kernel<Op><<<unsigned(nt), kScanThreads, 0, s>>>(op, n, tmp, out);
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Cell-table geometry for n cells per axis.
inline int bricks_per_axis(int n) { return (n + kBrick - 1) / kBrick; }
inline int64_t cell_table_entries(int n) {
    int64_t nb = bricks_per_axis(n);
    return nb * nb * nb * kBrickCells;
}

}  // namespace jfof

// Context (opaque in the C ABI).
namespace jfof {
struct Tracer;
struct BatchCache;
void destroy_batch_cache(BatchCache *);
struct TuneCache;
void destroy_tune_cache(TuneCache *);
}  // namespace jfof
struct jfof_ctx {
    jfof::Tracer *tracer; // null unless tracing is on
    jfof::BatchCache *batch; // cached graph of the last batched call
    int device;
    cudaStream_t stream;
    int *d_status;       // device status word
    int *h_status;       // pinned host mirror
    int64_t loop_budget;
    int dense_threshold;
    int small_threshold;
    int cta_shape;           // CTA shape of the list-driven link kernels (tuning knob)
    jfof::TuneCache *tune;   // autotuner choices per size bucket (first use)
    cudaStream_t copy_stream;  // velocity uploads of jfof_fof_host (created on first use)
    cudaEvent_t ev_pos, ev_vel;
    cudaStream_t cap_stream;        // capture stream of the REINFORCE sample graph (first use)
    cudaGraphExec_t sample_exec;    // that graph, updated in place between calls
    jfof::DevStatus dev() const { return jfof::DevStatus{d_status, loop_budget}; }
};

// ---------------------------------------------------------------------------
// Optional per-launch tracing: when a context has tracing on, every internal
// kernel launch is bracketed by two CUDA events recorded on the launching
// stream; jfof_trace_read aggregates elapsed time per kernel name.
namespace jfof {
struct Tracer;
extern thread_local Tracer *t_tracer;  // set for the duration of an ABI call
struct TraceScope {
    Tracer *tr;
    int idx;
    cudaStream_t s;
    TraceScope(const char *name, cudaStream_t s);
    ~TraceScope();
};
struct CtxScope {
    Tracer *prev;
    explicit CtxScope(jfof_ctx *c);
    ~CtxScope();
};
}  // namespace jfof
#define JFOF_CAT2(a, b) a##b
#define JFOF_CAT(a, b) JFOF_CAT2(a, b)
#define JFOF_TRACE(name, stream) jfof::TraceScope JFOF_CAT(jfof_trace_, __LINE__)(name, stream)
