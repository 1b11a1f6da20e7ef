// api.cu -- the C ABI (include/jfof.h): argument checks, workspace layout,
// launches on the context's stream, and the latched device status.
#include <atomic>
#include <cmath>
#include <cstring>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

using namespace jfof;

namespace jfof {

constexpr int32_t kMaxCellsPerAxis = 1600;

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

int check_box(int64_t N, float L, float b) {
    if (N < 1 || N > int64_t(INT32_MAX)) return JFOF_EINVAL;
    if (!finite_pos(L) || !finite_pos(b)) return JFOF_EINVAL;
    if (!(double(b) < 0.5 * double(L))) return JFOF_EINVAL;
    return JFOF_OK;
}

int32_t max_cells(float L, float b) {
    double m = std::floor(double(L) / (1.01 * double(b)));
    if (m < 1.0) m = 1.0;
    if (m > kMaxCellsPerAxis) m = kMaxCellsPerAxis;
    int32_t n = int32_t(m);
    if (n == 2) n = 1;
    return n;
}

int resolve_n(int64_t N, float L, float b, int32_t n_axis, int32_t *out) {
    int32_t nmax = max_cells(L, b);
    if (n_axis == 0) {
        int32_t n = nmax;
        while (n > 3 && double(n) * n * n > double(N)) --n;
        // When cells of that size are too wide for the sub-cell path of dense
        // cells (more than kSubSide sub-cells per side), take the next few
        // sizes up: one more cell per axis usually brings it back.
        const int32_t hi = n + (n / 8 > 2 ? n / 8 : 2);
        for (int32_t m = n; m <= hi && m <= nmax; ++m) {
            if (m < 5) break;
            if (make_link_params(N, L, b, m, kDefaultSmallThreshold, kDenseAuto).T > 0) {
                n = m;
                break;
            }
        }
        *out = n;
        return JFOF_OK;
    }
    if (n_axis < 0 || n_axis == 2 || n_axis > nmax) return JFOF_EINVAL;
    *out = n_axis;
    return JFOF_OK;
}

}  // namespace jfof

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? JFOF_OK : JFOF_ECUDA; }

int launch_status() { return cuda_status(cudaGetLastError()); }

}  // namespace

namespace jfof {

size_t fof_layout(int64_t N, int n, FofBuffers *fb, void *base) {
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    int64_t nb = bricks_per_axis(n);
    int64_t n_bricks = nb * nb * nb;
    FofBuffers f;
    f.spos = reinterpret_cast<float4 *>(take(sizeof(float4) * size_t(N)));
    f.cell_start = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(cell_table_entries(n) + 1)));
    f.brick_count = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(n_bricks + 1)));
    f.brick_start = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(n_bricks + 1)));
    f.cursor = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(n_bricks + 1)));
    const int64_t few = n_bricks <= kFewBricks ? n_bricks * kFewGrid : 0;
    f.scan_tmp = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * scan_tmp_words(few > n_bricks ? few : n_bricks)));
    f.bin_mat = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(few)));
    f.bin_base = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(few + 1)));
    // bin scatter buffer; dense-cell staging; then the link's rootmin[N]
    f.tmp = reinterpret_cast<float4 *>(take(sizeof(float4) * size_t(N)));
    f.parent = reinterpret_cast<int *>(take(sizeof(int) * size_t(N)));
    f.dense_id = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(cell_table_entries(n))));
    int64_t D_cap = dense_cap(N);
    f.dense_cells = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(D_cap)));
    f.counters = reinterpret_cast<uint32_t *>(take(kCounters * sizeof(uint32_t)));
    f.small_slots = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N)));
    f.sub_start = reinterpret_cast<uint16_t *>(take(sizeof(uint16_t) * size_t(D_cap) * (kSubMax + 1)));
    f.sub_rows = reinterpret_cast<uint16_t *>(take(sizeof(uint16_t) * size_t(D_cap) * (kSubSide * kSubSide)));
    f.medium_cells = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(medium_cap(N))));
    f.bucket_fill = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * kTailBuckets));
    if (fb) *fb = f;
    return off;
}

// SM count of the current device, queried once per device (GB300: 152).
int num_sms() {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    if (dev >= kMaxDevices) dev = kMaxDevices - 1;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

}  // namespace jfof

extern "C" {

const char *jfof_strerror(int code) {
    switch (code) {
        case JFOF_OK: return "ok";
        case JFOF_EINVAL: return "invalid argument";
        case JFOF_ERANGE: return "position outside [0, L) (or not finite) without JFOF_WRAP";
        case JFOF_ENOMEM: return "workspace too small";
        case JFOF_ECUDA: return "CUDA runtime error";
        case JFOF_ETIMEOUT: return "bounded device loop ran out of iterations";
        case JFOF_EOVERFLOW: return "output capacity too small";
        default: return "unknown status";
    }
}

int jfof_create(jfof_ctx **ctx, int device, void *stream) {
    if (!ctx) return JFOF_EINVAL;
    *ctx = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return JFOF_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
        return JFOF_ECUDA;
    (void)num_sms();  // launch grids are sized by this device's SM count from here on
    jfof_ctx *c = new jfof_ctx();
    c->device = device;
    c->tracer = nullptr;
    c->batch = nullptr;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->loop_budget = kDefaultLoopBudget;
    c->dense_threshold = kDenseAuto;
    c->small_threshold = kDefaultSmallThreshold;
    c->cta_shape = 0;
    c->tune = nullptr;
    c->copy_stream = nullptr;
    c->ev_pos = nullptr;
    c->ev_vel = nullptr;
    c->cap_stream = nullptr;
    c->sample_exec = nullptr;
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess) {
        delete c;
        return JFOF_ECUDA;
    }
    if (cudaMallocHost(&c->h_status, sizeof(int)) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return JFOF_ECUDA;
    }
    *c->h_status = 0;
    if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(c->d_status);
        cudaFreeHost(c->h_status);
        delete c;
        return JFOF_ECUDA;
    }
    *ctx = c;
    return JFOF_OK;
}

int jfof_destroy(jfof_ctx *ctx) {
    if (!ctx) return JFOF_EINVAL;
    jfof_trace_enable(ctx, 0);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    destroy_batch_cache(ctx->batch);
    destroy_tune_cache(ctx->tune);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaEventDestroy(ctx->ev_pos);
        cudaEventDestroy(ctx->ev_vel);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->sample_exec) cudaGraphExecDestroy(ctx->sample_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    delete ctx;
    return JFOF_OK;
}

int jfof_set_stream(jfof_ctx *ctx, void *stream) {
    if (!ctx) return JFOF_EINVAL;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    return JFOF_OK;
}

int jfof_set_loop_budget(jfof_ctx *ctx, int64_t iterations) {
    if (!ctx || iterations < 0) return JFOF_EINVAL;
    ctx->loop_budget = iterations == 0 ? kDefaultLoopBudget : iterations;
    return JFOF_OK;
}

int jfof_sync(jfof_ctx *ctx) {
    if (!ctx) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    if (cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return JFOF_ECUDA;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return JFOF_ECUDA;
    int st = *ctx->h_status;
    if (st != 0) cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
    return st;
}

int jfof_max_cells_per_axis(float L, float b, int32_t *n_axis) {
    if (!n_axis || !finite_pos(L) || !finite_pos(b)) return JFOF_EINVAL;
    *n_axis = max_cells(L, b);
    return JFOF_OK;
}

int jfof_default_cells_per_axis(int64_t N, float L, float b, int32_t *n_axis) {
    if (!n_axis) return JFOF_EINVAL;
    int e = check_box(N, L, b);
    if (e) return e;
    return resolve_n(N, L, b, 0, n_axis);
}

int jfof_fof_bytes(int64_t N, int32_t n_axis, size_t *bytes) {
    if (!bytes || N < 1 || N > int64_t(INT32_MAX) || n_axis < 1 || n_axis == 2 || n_axis > kMaxCellsPerAxis)
        return JFOF_EINVAL;
    *bytes = fof_layout(N, n_axis, nullptr, nullptr);
    return JFOF_OK;
}

int jfof_bin_cells(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, int32_t n_axis, uint32_t flags,
                   void *ws, size_t ws_bytes, jfof_cells *cells) {
    if (!ctx || !pos || !ws || !cells) return JFOF_EINVAL;
    int e = check_box(N, L, b);
    if (e) return e;
    int32_t n;
    if ((e = resolve_n(N, L, b, n_axis, &n))) return e;
    FofBuffers fb;
    size_t need = fof_layout(N, n, &fb, ws);
    if (ws_bytes < need) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    LinkParams lp = make_link_params(N, L, b, n, ctx->small_threshold, ctx->dense_threshold, ctx->cta_shape);
    launch_bin_cells(pos, N, L, n, (flags & JFOF_WRAP) != 0, lp, fb, ctx->dev(), ctx->stream);
    jfof_cells c;
    c.n = N;
    c.n_axis = n;
    c.brick = kBrick;
    c.L = L;
    c.b = b;
    c.flags = flags;
    c.small_threshold = lp.S;
    c.dense_threshold = lp.T;
    c.spos = fb.spos;
    c.cell_start = fb.cell_start;
    c.n_cells_table = cell_table_entries(n);
    c.workspace = ws;
    *cells = c;
    return launch_status();
}

int jfof_link(jfof_ctx *ctx, const jfof_cells *cells, int32_t *label) {
    if (!ctx || !cells || !label || !cells->spos || !cells->cell_start || !cells->workspace) return JFOF_EINVAL;
    int e = check_box(cells->n, cells->L, cells->b);
    if (e) return e;
    if (cells->n_axis < 1 || cells->n_axis == 2 || cells->n_axis > max_cells(cells->L, cells->b)) return JFOF_EINVAL;
    FofBuffers fb;
    fof_layout(cells->n, cells->n_axis, &fb, cells->workspace);
    if (fb.spos != cells->spos || fb.cell_start != cells->cell_start) return JFOF_EINVAL;
    LinkParams lp = make_link_params(cells->n, cells->L, cells->b, cells->n_axis, cells->small_threshold,
                                     cells->dense_threshold, ctx->cta_shape);
    if (lp.T != cells->dense_threshold || lp.S != cells->small_threshold) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_link(*cells, fb, lp, label, ctx->dev(), ctx->stream);
    return launch_status();
}

int jfof_set_cta_shape(jfof_ctx *ctx, int32_t shape) {
    if (!ctx || shape < 0 || shape >= kCtaShapes) return JFOF_EINVAL;
    ctx->cta_shape = shape;
    return JFOF_OK;
}

int jfof_set_cell_classes(jfof_ctx *ctx, int32_t small_max, int32_t dense_over) {
    if (!ctx || small_max < 0 || dense_over < kDenseAuto) return JFOF_EINVAL;
    ctx->small_threshold = small_max;
    ctx->dense_threshold = dense_over;
    return JFOF_OK;
}

int jfof_groups_bytes(int64_t N, size_t *bytes) {
    if (!bytes || N < 1 || N > int64_t(INT32_MAX)) return JFOF_EINVAL;
    *bytes = groups_layout(N, N, nullptr, nullptr);
    return JFOF_OK;
}

int jfof_groups(jfof_ctx *ctx, const int32_t *label, int64_t N, int32_t min_size, void *ws, size_t ws_bytes,
                int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members, int32_t *n_halos) {
    if (!ctx || !label || !ws || !halo_id || !count || !halo_start || !members || !n_halos) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX) || min_size < 1) return JFOF_EINVAL;
    int64_t H_cap = N / min_size;
    if (H_cap < 1) H_cap = 1;
    GroupBuffers gb;
    size_t need = groups_layout(N, H_cap, &gb, ws);
    if (ws_bytes < need) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_groups(label, N, min_size, H_cap, gb, halo_id, count, halo_start, members, n_halos, ctx->dev(),
                  ctx->stream);
    return launch_status();
}

int jfof_halo_props(jfof_ctx *ctx, const float *pos, const float *vel, int64_t N, float L, uint32_t flags,
                    const int32_t *halo_start, const int32_t *members, const int32_t *n_halos, int64_t H_cap,
                    float particle_mass, float *mass, float *com, float *vmean, float *sigv) {
    if (!ctx || !pos || !halo_start || !members || !n_halos || !mass || !com) return JFOF_EINVAL;
    if (vel && (!vmean || !sigv)) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX) || H_cap < 1 || !finite_pos(L)) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_halo_props(pos, vel, N, L, (flags & JFOF_WRAP) != 0, halo_start, members, n_halos, H_cap, particle_mass,
                      mass, com, vmean, sigv, ctx->stream);
    return launch_status();
}

int jfof_halo_props_backward(jfof_ctx *ctx, const float *vel, const int32_t *halo_id, const int32_t *count,
                             int64_t N, const float *vmean, const float *sigv, const float *g_com,
                             const float *g_vmean, const float *g_sigv, float *g_pos, float *g_vel) {
    if (!ctx || !halo_id || !count) return JFOF_EINVAL;
    if (g_sigv && (!vel || !vmean || !sigv)) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX)) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_halo_props_backward(vel, halo_id, count, N, vmean, sigv, g_com, g_vmean, g_sigv, g_pos, g_vel,
                               ctx->stream);
    return launch_status();
}

int jfof_fof_all_bytes(int64_t N, int32_t n_axis, size_t *bytes) {
    size_t a, g;
    int e = jfof_fof_bytes(N, n_axis, &a);
    if (e) return e;
    if ((e = jfof_groups_bytes(N, &g))) return e;
    *bytes = a + g;
    return JFOF_OK;
}

int jfof_fof(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, int32_t n_axis, uint32_t flags,
             int32_t min_size, void *ws, size_t ws_bytes, int32_t *label, int32_t *halo_id, int32_t *count,
             int32_t *halo_start, int32_t *members, int32_t *n_halos) {
    if (!ctx || !ws || !label || !halo_id || !count || !halo_start || !members || !n_halos || min_size < 1)
        return JFOF_EINVAL;
    int e = check_box(N, L, b);
    if (e) return e;
    int32_t n;
    if ((e = resolve_n(N, L, b, n_axis, &n))) return e;
    size_t a = fof_layout(N, n, nullptr, nullptr);
    size_t g;
    jfof_groups_bytes(N, &g);
    if (ws_bytes < a + g) return JFOF_ENOMEM;
    jfof_cells cells;
    if ((e = jfof_bin_cells(ctx, pos, N, L, b, n, flags, ws, a, &cells))) return e;
    // link, then labels and groups straight from the forest
    int64_t H_cap = N / min_size;
    if (H_cap < 1) H_cap = 1;
    FofBuffers fb;
    fof_layout(N, n, &fb, ws);
    GroupBuffers gb;
    groups_layout(N, H_cap, &gb, reinterpret_cast<char *>(ws) + a);
    LinkParams lp = make_link_params(N, L, b, n, cells.small_threshold, cells.dense_threshold, ctx->cta_shape);
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_link_core(cells, fb, lp, ctx->dev(), ctx->stream);
    launch_tail_groups(fb, N, min_size, H_cap, gb, label, halo_id, count, halo_start, members, n_halos,
                       ctx->stream);
    return launch_status();
}

}  // extern "C"
