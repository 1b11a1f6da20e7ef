// api_reinforce.cu -- C ABI of the REINFORCE topological mode (a11-a13) and
// the verification hooks (include/jfof.h).
#include <cmath>

#include "jfof_internal.cuh"
#include "k_fof.cuh"
#include "k_reinforce.cuh"

using namespace jfof;

namespace {

bool pos_finite(float x) { return std::isfinite(x) && x > 0.0f; }

// Pair-cut grid: the largest legal n (cells >= 1.01 r_cut) with n^3 <= N.
int pair_grid(int64_t N, float L, float r_cut) {
    double m = std::floor(double(L) / (1.01 * double(r_cut)));
    if (m < 1.0) m = 1.0;
    if (m > 1600.0) m = 1600.0;
    int n = int(m);
    while (n > 3 && double(n) * n * n > double(N)) --n;
    if (n == 2) n = 1;
    return n;
}

int status_of_launch() { return cudaGetLastError() == cudaSuccess ? JFOF_OK : JFOF_ECUDA; }

}  // namespace

extern "C" {

int jfof_prob_coef(float b, int32_t prob_form, float tau, float alpha, float *coef) {
    if (!coef || !pos_finite(b) || (prob_form != 0 && prob_form != 1)) return JFOF_EINVAL;
    if (prob_form == 0) {
        double t = tau > 0.0f ? double(tau) : 0.05 * double(b);
        *coef = float(1.0 / t);
    } else {
        float b2 = host_mul(b, b);
        *coef = float(double(alpha) / double(b2));
    }
    return JFOF_OK;
}

int jfof_pairs_bytes(int64_t N, float L, float r_cut, size_t *bytes) {
    if (!bytes || N < 1 || N > int64_t(INT32_MAX) || !pos_finite(L) || !pos_finite(r_cut)) return JFOF_EINVAL;
    *bytes = pairs_layout(N, pair_grid(N, L, r_cut), nullptr, nullptr);
    return JFOF_OK;
}

int jfof_pairs(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, float r_cut, int32_t prob_form,
               float coef, uint32_t flags, void *ws, size_t ws_bytes, int64_t cap, int32_t *pair_i, int32_t *pair_j,
               float *pair_d, float *pair_p, int64_t *n_pairs) {
    if (!ctx || !pos || !ws || !n_pairs || cap < 0) return JFOF_EINVAL;
    if (cap > 0 && (!pair_i || !pair_j || !pair_d || !pair_p)) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX) || !pos_finite(L) || !pos_finite(b) || !pos_finite(r_cut)) return JFOF_EINVAL;
    if (!(double(r_cut) < 0.5 * double(L)) || (prob_form != 0 && prob_form != 1) || !std::isfinite(coef))
        return JFOF_EINVAL;
    int n = pair_grid(N, L, r_cut);
    PairBuffers pb;
    size_t need = pairs_layout(N, n, &pb, ws);
    if (ws_bytes < need) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    float rc2 = host_mul(r_cut, r_cut), b2 = host_mul(b, b);
    PairGeom pg{L, 0.5f * L, rc2, b, b2, coef, float(double(n) / double(L)), n, bricks_per_axis(n), prob_form,
                (flags & JFOF_WRAP) != 0};
    launch_pairs(pos, N, pg, pb, cap, pair_i, pair_j, pair_d, pair_p, n_pairs, ctx->dev(), ctx->stream);
    return status_of_launch();
}

int jfof_reinforce_sample_bytes(int64_t N, size_t *bytes) {
    if (!bytes || N < 1 || N > int64_t(INT32_MAX)) return JFOF_EINVAL;
    *bytes = sample_layout(N, nullptr, nullptr);
    return JFOF_OK;
}

int jfof_reinforce_sample(jfof_ctx *ctx, int64_t N, const int32_t *pair_i, const int32_t *pair_j,
                          const float *pair_p, int64_t E, int32_t K, uint64_t seed, int32_t min_size, void *ws,
                          size_t ws_bytes, int32_t *labels, int32_t *n_halos) {
    if (!ctx || !ws || !labels || !n_halos || N < 1 || N > int64_t(INT32_MAX) || E < 0 || K < 1 || min_size < 1)
        return JFOF_EINVAL;
    if (E > 0 && (!pair_i || !pair_j || !pair_p)) return JFOF_EINVAL;
    uint32_t *counts;
    if (ws_bytes < sample_layout(N, &counts, ws)) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    // All K samples (chunks of kSampleChunk, four launches each) as one CUDA
    // graph launched on the context's stream.  It is captured on a
    // library-owned stream (the caller's may be the legacy default stream,
    // which cannot be captured); a later call with the same shape updates the
    // instantiated graph's parameters (seed, pointers) in place.
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return JFOF_ECUDA;
    Tracer *tr = t_tracer;
    t_tracer = nullptr;  // no per-launch trace events inside the capture
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        t_tracer = tr;
        return JFOF_ECUDA;
    }
    launch_reinforce_sample(N, pair_i, pair_j, pair_p, E, K, seed, min_size, counts, labels, n_halos, ctx->dev(),
                            ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    t_tracer = tr;
    if (ce != cudaSuccess) return JFOF_ECUDA;
    if (ctx->sample_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ctx->sample_exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();  // a different shape: instantiate anew
            cudaGraphExecDestroy(ctx->sample_exec);
            ctx->sample_exec = nullptr;
        }
    }
    if (!ctx->sample_exec && cudaGraphInstantiate(&ctx->sample_exec, graph, 0) != cudaSuccess) {
        ctx->sample_exec = nullptr;
        cudaGraphDestroy(graph);
        return JFOF_ECUDA;
    }
    cudaGraphDestroy(graph);
    {
        JFOF_TRACE("reinforce_sample", ctx->stream);
        if (cudaGraphLaunch(ctx->sample_exec, ctx->stream) != cudaSuccess) return JFOF_ECUDA;
    }
    return status_of_launch();
}

int jfof_reinforce_grad_bytes(int64_t N, int64_t E, size_t *bytes) {
    if (!bytes || N < 1 || N > int64_t(INT32_MAX) || E < 0 || E > int64_t(UINT32_MAX)) return JFOF_EINVAL;
    *bytes = grad_layout(N, E, nullptr, nullptr);
    return JFOF_OK;
}

int jfof_reinforce_grad(jfof_ctx *ctx, const float *pos, int64_t N, float L, uint32_t flags, const int32_t *pair_i,
                        const int32_t *pair_j, const float *pair_d, const float *pair_p, int64_t E, int32_t K,
                        uint64_t seed, const float *advantage, int32_t prob_form, float coef, void *ws,
                        size_t ws_bytes, float *g_pos) {
    if (!ctx || !pos || !advantage || !ws || !g_pos || N < 1 || N > int64_t(INT32_MAX) || K < 1) return JFOF_EINVAL;
    if (E < 0 || E > int64_t(UINT32_MAX) || (E > 0 && (!pair_i || !pair_j || !pair_d || !pair_p))) return JFOF_EINVAL;
    if (!pos_finite(L) || (prob_form != 0 && prob_form != 1)) return JFOF_EINVAL;
    GradBuffers gb;
    if (ws_bytes < grad_layout(N, E, &gb, ws)) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_reinforce_grad(pos, N, L, (flags & JFOF_WRAP) != 0, pair_i, pair_j, pair_d, pair_p, E, K, seed,
                          advantage, prob_form, coef, gb, g_pos, ctx->stream);
    return status_of_launch();
}

int jfof_eval_exp(jfof_ctx *ctx, const float *x, float *y, int64_t n) {
    if (!ctx || !x || !y || n < 0) return JFOF_EINVAL;
    if (n == 0) return JFOF_OK;
    cudaSetDevice(ctx->device);
    launch_eval_exp(x, y, n, ctx->stream);
    return status_of_launch();
}

int jfof_eval_edge_uniform(jfof_ctx *ctx, uint64_t seed, const int32_t *i, const int32_t *j, const int32_t *k,
                           float *u, int64_t n) {
    if (!ctx || !i || !j || !k || !u || n < 0) return JFOF_EINVAL;
    if (n == 0) return JFOF_OK;
    cudaSetDevice(ctx->device);
    launch_eval_uniform(seed, i, j, k, u, n, ctx->stream);
    return status_of_launch();
}

}  // extern "C"
