// api_batch.cu -- a10: many independent boxes of uneven size in one CUDA-graph
// launch (each box's bin/link/groups pipeline on its own stream branch, so
// small boxes and the narrow phases of large ones overlap), the per-box loop
// it is compared with, and the autotuner (grid size, cell classes and CTA
// shape of the link kernels, with a per-size-bucket cache in the context).
#include <cmath>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

using namespace jfof;

namespace jfof {

// One box: bin, link and groups on stream s, all buffers in ws.
struct BoxPlan {
    int64_t N;
    float L, b;
    int n;
    LinkParams lp;
    int64_t H_cap;
    size_t ws_off, fof_bytes, grp_bytes;
    size_t count_off, start_off, members_off, total;
};

static BoxPlan plan_box(int64_t N, float L, float b, int n, int S, int T, int shape, int min_size) {
    BoxPlan p{};
    p.N = N;
    p.L = L;
    p.b = b;
    p.n = n;
    p.lp = make_link_params(N, L, b, n, S, T, shape);
    p.H_cap = N / min_size > 0 ? N / min_size : 1;
    p.fof_bytes = fof_layout(N, n, nullptr, nullptr);
    p.grp_bytes = groups_layout(N, p.H_cap, nullptr, nullptr);
    p.count_off = p.fof_bytes + p.grp_bytes;
    p.start_off = p.count_off + align_up(sizeof(int32_t) * size_t(p.H_cap));
    p.members_off = p.start_off + align_up(sizeof(int32_t) * size_t(p.H_cap + 1));
    p.total = p.members_off + align_up(sizeof(int32_t) * size_t(N));
    return p;
}

static void run_box(const BoxPlan &p, const float *pos, uint32_t flags, int min_size, char *ws, int32_t *label,
                    int32_t *halo_id, int32_t *n_halos, const DevStatus &st, cudaStream_t s) {
    FofBuffers fb;
    fof_layout(p.N, p.n, &fb, ws);
    launch_bin_cells(pos, p.N, p.L, p.n, (flags & JFOF_WRAP) != 0, p.lp, fb, st, s);
    jfof_cells c{};
    c.n = p.N;
    c.n_axis = p.n;
    c.brick = kBrick;
    c.L = p.L;
    c.b = p.b;
    c.flags = flags;
    c.small_threshold = p.lp.S;
    c.dense_threshold = p.lp.T;
    c.spos = fb.spos;
    c.cell_start = fb.cell_start;
    c.n_cells_table = cell_table_entries(p.n);
    c.workspace = ws;
    launch_link_core(c, fb, p.lp, st, s);
    GroupBuffers gb;
    groups_layout(p.N, p.H_cap, &gb, ws + p.fof_bytes);
    launch_tail_groups(fb, p.N, min_size, p.H_cap, gb, label, halo_id, reinterpret_cast<int32_t *>(ws + p.count_off),
                       reinterpret_cast<int32_t *>(ws + p.start_off), reinterpret_cast<int32_t *>(ws + p.members_off),
                       n_halos, s);
}

// Cached graph of the last batch configuration.
struct BatchCache {
    std::vector<int64_t> off;
    std::vector<float> L, b;
    std::vector<int> n, S, T, W;
    const void *pos = nullptr, *ws = nullptr, *label = nullptr, *halo_id = nullptr, *n_halos = nullptr;
    uint32_t flags = 0;
    int min_size = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> streams;  // [0] capture origin, [1..B] box branches
    std::vector<cudaEvent_t> events;    // [0] fork, [1..B] joins
    ~BatchCache() {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto s : streams) cudaStreamDestroy(s);
        for (auto e : events) cudaEventDestroy(e);
    }
};

void destroy_batch_cache(BatchCache *c) { delete c; }

// Autotuner choices by size bucket: (round(2 log2 N), round(4 log2(L/b))).
struct TuneChoice {
    double n_ratio;  // chosen n over the default n of the box
    int S, T, shape;
    float ms;
};
struct TuneCache {
    std::map<std::pair<int, int>, TuneChoice> best;
};

void destroy_tune_cache(TuneCache *c) { delete c; }

}  // namespace jfof

namespace {

struct BatchArgs {
    int64_t total_N;
    std::vector<BoxPlan> boxes;
    size_t ws_bytes;
};

int plan_batch(const int64_t *h_off, int32_t B, const float *h_L, const float *h_b, const int32_t *h_n,
               const int32_t *h_S, const int32_t *h_T, const int32_t *h_W, int S_def, int T_def, int W_def,
               int min_size, BatchArgs *out) {
    if (!h_off || B < 1 || !h_L || !h_b || min_size < 1 || h_off[0] != 0) return JFOF_EINVAL;
    out->boxes.clear();
    size_t off = 0;
    for (int k = 0; k < B; ++k) {
        int64_t N = h_off[k + 1] - h_off[k];
        int e = check_box(N, h_L[k], h_b[k]);
        if (e) return e;
        int32_t n;
        if ((e = resolve_n(N, h_L[k], h_b[k], h_n ? h_n[k] : 0, &n))) return e;
        const int W = h_W ? h_W[k] : W_def;
        if (W < 0 || W >= kCtaShapes) return JFOF_EINVAL;
        BoxPlan p = plan_box(N, h_L[k], h_b[k], n, h_S ? h_S[k] : S_def, h_T ? h_T[k] : T_def, W, min_size);
        p.ws_off = off;
        off += align_up(p.total);
        out->boxes.push_back(p);
    }
    out->total_N = h_off[B];
    if (out->total_N > int64_t(INT32_MAX)) return JFOF_EINVAL;
    out->ws_bytes = off;
    return JFOF_OK;
}

bool same_config(const BatchCache &c, const BatchArgs &a, const int64_t *h_off, int32_t B, const float *pos,
                 const void *ws, const int32_t *label, const int32_t *halo_id, const int32_t *n_halos,
                 uint32_t flags, int min_size, cudaStream_t stream) {
    if (!c.exec || int(c.n.size()) != B || c.pos != pos || c.ws != ws || c.label != label ||
        c.halo_id != halo_id || c.n_halos != n_halos || c.flags != flags || c.min_size != min_size ||
        c.stream != stream)
        return false;
    for (int k = 0; k < B; ++k) {
        const BoxPlan &p = a.boxes[k];
        if (c.off[k + 1] != h_off[k + 1] || c.L[k] != p.L || c.b[k] != p.b || c.n[k] != p.n || c.S[k] != p.lp.S ||
            c.T[k] != p.lp.T || c.W[k] != p.lp.warps[0] * 100 + p.lp.warps[1] * 10 + p.lp.warps[2])
            return false;
    }
    return true;
}

}  // namespace

extern "C" {

int jfof_batch_bytes(const int64_t *h_box_offset, int32_t B, const float *h_L, const float *h_b,
                     const int32_t *h_n_axis, int32_t min_size, size_t *bytes) {
    if (!bytes) return JFOF_EINVAL;
    BatchArgs a;
    int e = plan_batch(h_box_offset, B, h_L, h_b, h_n_axis, nullptr, nullptr, nullptr, 8, 64, 0, min_size, &a);
    if (e) return e;
    *bytes = a.ws_bytes;
    return JFOF_OK;
}

int jfof_fof_batched(jfof_ctx *ctx, const float *pos, const int64_t *h_box_offset, int32_t B, const float *h_L,
                     const float *h_b, const int32_t *h_n_axis, const int32_t *h_small, const int32_t *h_dense,
                     const int32_t *h_shape, uint32_t flags, int32_t min_size, void *ws, size_t ws_bytes,
                     int32_t *label, int32_t *halo_id, int32_t *n_halos, int32_t use_graph) {
    if (!ctx || !pos || !ws || !label || !halo_id || !n_halos) return JFOF_EINVAL;
    BatchArgs a;
    int e = plan_batch(h_box_offset, B, h_L, h_b, h_n_axis, h_small, h_dense, h_shape, ctx->small_threshold,
                       ctx->dense_threshold, ctx->cta_shape, min_size, &a);
    if (e) return e;
    if (ws_bytes < a.ws_bytes) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    char *base = reinterpret_cast<char *>(ws);
    DevStatus st = ctx->dev();
    if (!use_graph) {
        CtxScope scope(ctx);
        for (int k = 0; k < B; ++k) {
            const BoxPlan &p = a.boxes[k];
            int64_t o = h_box_offset[k];
            run_box(p, pos + 3 * o, flags, min_size, base + p.ws_off, label + o, halo_id + o, n_halos + k, st,
                    ctx->stream);
        }
        return cudaGetLastError() == cudaSuccess ? JFOF_OK : JFOF_ECUDA;
    }
    if (!ctx->batch) ctx->batch = new BatchCache();
    BatchCache &c = *ctx->batch;
    if (!same_config(c, a, h_box_offset, B, pos, ws, label, halo_id, n_halos, flags, min_size, ctx->stream)) {
        if (c.exec) {
            cudaGraphExecDestroy(c.exec);
            c.exec = nullptr;
        }
        while (int(c.streams.size()) < B + 1) {
            cudaStream_t s;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return JFOF_ECUDA;
            c.streams.push_back(s);
        }
        while (int(c.events.size()) < B + 1) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return JFOF_ECUDA;
            c.events.push_back(ev);
        }
        // capture on a library-owned stream (the caller's may be the legacy
        // default stream, which cannot be captured): fork, one branch per box,
        // join; the graph is then launched on the caller's stream
        cudaStream_t origin = c.streams[0];
        jfof::t_tracer = nullptr;
        if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return JFOF_ECUDA;
        cudaEventRecord(c.events[0], origin);
        for (int k = 0; k < B; ++k) {
            const BoxPlan &p = a.boxes[k];
            int64_t o = h_box_offset[k];
            cudaStreamWaitEvent(c.streams[k + 1], c.events[0], 0);
            run_box(p, pos + 3 * o, flags, min_size, base + p.ws_off, label + o, halo_id + o, n_halos + k, st,
                    c.streams[k + 1]);
            cudaEventRecord(c.events[k + 1], c.streams[k + 1]);
            cudaStreamWaitEvent(origin, c.events[k + 1], 0);
        }
        cudaGraph_t graph;
        if (cudaStreamEndCapture(origin, &graph) != cudaSuccess) return JFOF_ECUDA;
        cudaError_t ie = cudaGraphInstantiate(&c.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            c.exec = nullptr;
            return JFOF_ECUDA;
        }
        c.off.assign(h_box_offset, h_box_offset + B + 1);
        c.L.clear();
        c.b.clear();
        c.n.clear();
        c.S.clear();
        c.T.clear();
        c.W.clear();
        for (auto &p : a.boxes) {
            c.L.push_back(p.L);
            c.b.push_back(p.b);
            c.n.push_back(p.n);
            c.S.push_back(p.lp.S);
            c.T.push_back(p.lp.T);
            c.W.push_back(p.lp.warps[0] * 100 + p.lp.warps[1] * 10 + p.lp.warps[2]);
        }
        c.pos = pos;
        c.ws = ws;
        c.label = label;
        c.halo_id = halo_id;
        c.n_halos = n_halos;
        c.flags = flags;
        c.min_size = min_size;
        c.stream = ctx->stream;
    }
    return cudaGraphLaunch(c.exec, ctx->stream) == cudaSuccess ? JFOF_OK : JFOF_ECUDA;
}

// Autotuner: times jfof_fof-equivalent runs of one box (one warm-up, then
// `reps` runs each, CUDA events) over grids n in {n0, 0.8 n0, 1.26 n0}
// (those whose workspace fits ws) and six cell-class pairs (S, T) with the
// default CTA shape, then the other CTA shapes of the link kernels for the
// best of those, and returns the fastest.  The choice is kept in the context
// by size bucket (round(2 log2 N), round(4 log2(L/b))); with use_cache a box
// of a known bucket gets it back without timing (*best_ms = the time it was
// chosen with).  With a flush buffer (larger than L2), each timed run starts
// after the buffer is overwritten, so a small box is timed with its data in
// DRAM as it would be inside a batch, not resident in L2 from the run before.
// Synchronises.  Labels do not depend on the choice.
int jfof_autotune(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, uint32_t flags, int32_t min_size,
                  void *ws, size_t ws_bytes, int32_t *label, int32_t *halo_id, int32_t *n_halos, int32_t reps,
                  int32_t use_cache, void *flush, size_t flush_bytes, int32_t *best_n_axis, int32_t *best_small,
                  int32_t *best_dense, int32_t *best_shape, float *best_ms) {
    if (!ctx || !pos || !ws || !label || !halo_id || !n_halos || !best_n_axis || !best_small || !best_dense ||
        !best_shape || reps < 1)
        return JFOF_EINVAL;
    int e = check_box(N, L, b);
    if (e) return e;
    int32_t n0;
    if ((e = resolve_n(N, L, b, 0, &n0))) return e;
    int32_t nmax = max_cells(L, b);
    const std::pair<int, int> key{int(std::lround(2.0 * std::log2(double(N)))),
                                  int(std::lround(4.0 * std::log2(double(L) / double(b))))};
    if (!ctx->tune) ctx->tune = new TuneCache();
    auto legal = [&](int n) { return n >= 3 && n <= nmax; };
    if (use_cache) {
        auto it = ctx->tune->best.find(key);
        if (it != ctx->tune->best.end()) {
            const TuneChoice &c = it->second;
            int n = int(std::lround(n0 * c.n_ratio));
            if (!legal(n)) n = n0;
            BoxPlan p = plan_box(N, L, b, n, c.S, c.T, c.shape, min_size);
            if (p.total <= ws_bytes) {
                *best_n_axis = n;
                *best_small = c.S;
                *best_dense = c.T;
                *best_shape = c.shape;
                if (best_ms) *best_ms = c.ms;
                return JFOF_OK;
            }
        }
    }
    std::vector<int> ns = {n0};
    for (double f : {0.8, 1.26}) {
        int n = int(n0 * f);
        if (legal(n) && n != n0) ns.push_back(n);
    }
    const int dT = default_dense_threshold(N);
    const int cls[][2] = {{kDefaultSmallThreshold, dT}, {8, 96}, {16, 96}, {16, 128}, {16, 160}, {24, 128}};
    cudaSetDevice(ctx->device);
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess) return JFOF_ECUDA;
    if (cudaEventCreate(&t1) != cudaSuccess) {
        cudaEventDestroy(t0);
        return JFOF_ECUDA;
    }
    float best = 1e30f;
    int bn = n0, bS = kDefaultSmallThreshold, bT = dT, bW = 0;
    DevStatus st = ctx->dev();
    auto time_one = [&](int n, int S, int T, int W, float *ms) -> int {
        BoxPlan p = plan_box(N, L, b, n, S, T, W, min_size);
        if (p.total > ws_bytes) return 1;
        run_box(p, pos, flags, min_size, reinterpret_cast<char *>(ws), label, halo_id, n_halos, st, ctx->stream);
        float tot = 0.f;
        for (int r = 0; r < reps; ++r) {
            if (flush && flush_bytes) cudaMemsetAsync(flush, r & 0xff, flush_bytes, ctx->stream);
            cudaEventRecord(t0, ctx->stream);
            run_box(p, pos, flags, min_size, reinterpret_cast<char *>(ws), label, halo_id, n_halos, st, ctx->stream);
            cudaEventRecord(t1, ctx->stream);
            if (cudaEventSynchronize(t1) != cudaSuccess) return -1;
            float one = 0.f;
            cudaEventElapsedTime(&one, t0, t1);
            tot += one;
        }
        *ms = tot / reps;
        return 0;
    };
    int rc = 0;
    for (int n : ns)
        for (auto &c : cls) {
            float ms = 0.f;
            if ((rc = time_one(n, c[0], c[1], 0, &ms)) < 0) break;
            if (rc == 0 && ms < best) {
                best = ms;
                bn = n;
                bS = c[0];
                bT = c[1];
            }
        }
    for (int W = 1; W < kCtaShapes && rc >= 0 && best < 1e30f; ++W) {
        float ms = 0.f;
        if ((rc = time_one(bn, bS, bT, W, &ms)) < 0) break;
        if (rc == 0 && ms < best) {
            best = ms;
            bW = W;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc < 0) return JFOF_ECUDA;
    if (!(best < 1e30f)) return JFOF_ENOMEM;
    *best_n_axis = bn;
    *best_small = bS;
    *best_dense = bT;
    *best_shape = bW;
    if (best_ms) *best_ms = best;
    ctx->tune->best[key] = TuneChoice{double(bn) / double(n0), bS, bT, bW, best};
    return JFOF_OK;
}

}  // extern "C"
