// trace.cu -- per-kernel CUDA-event tracing for the ABI (jfof_trace_*).
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "jfof_internal.cuh"

namespace jfof {

struct Tracer {
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
};

thread_local Tracer *t_tracer = nullptr;

TraceScope::TraceScope(const char *name, cudaStream_t st) : tr(t_tracer), idx(-1), s(st) {
    if (!tr) return;
    Tracer::Rec r{name, tr->get(), tr->get()};
    cudaEventRecord(r.a, s);
    tr->recs.push_back(r);
    idx = int(tr->recs.size()) - 1;
}

TraceScope::~TraceScope() {
    if (tr && idx >= 0) cudaEventRecord(tr->recs[idx].b, s);
}

CtxScope::CtxScope(jfof_ctx *c) : prev(t_tracer) { t_tracer = c ? c->tracer : nullptr; }
CtxScope::~CtxScope() { t_tracer = prev; }

}  // namespace jfof

extern "C" {

int jfof_trace_enable(jfof_ctx *ctx, int on) {
    if (!ctx) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    if (on && !ctx->tracer) ctx->tracer = new jfof::Tracer();
    if (!on && ctx->tracer) {
        cudaStreamSynchronize(ctx->stream);
        for (auto &r : ctx->tracer->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : ctx->tracer->pool) cudaEventDestroy(e);
        delete ctx->tracer;
        ctx->tracer = nullptr;
    }
    return JFOF_OK;
}

int jfof_trace_read(jfof_ctx *ctx, char *buf, size_t len, size_t *written) {
    if (!ctx || !buf || len == 0) return JFOF_EINVAL;
    buf[0] = 0;
    if (written) *written = 0;
    if (!ctx->tracer) return JFOF_OK;
    cudaSetDevice(ctx->device);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return JFOF_ECUDA;
    std::map<std::string, std::pair<long, double>> agg;
    std::vector<std::string> order;
    for (auto &r : ctx->tracer->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            agg[r.name] = {1, double(ms)};
        } else {
            it->second.first += 1;
            it->second.second += ms;
        }
        ctx->tracer->pool.push_back(r.a);
        ctx->tracer->pool.push_back(r.b);
    }
    ctx->tracer->recs.clear();
    size_t off = 0;
    for (auto &name : order) {
        auto &v = agg[name];
        int k = snprintf(buf + off, len - off, "%s %ld %.6f\n", name.c_str(), v.first, v.second);
        if (k < 0 || size_t(k) >= len - off) return JFOF_EOVERFLOW;
        off += size_t(k);
    }
    if (written) *written = off;
    return JFOF_OK;
}

}  // extern "C"
