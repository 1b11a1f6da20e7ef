// api_host.cu -- jfof_fof_host: one step of the plain path (a1-a8) from host
// buffers.  Positions are uploaded on the context's stream; velocities on a
// library-owned copy stream once the positions are in, so their upload runs
// under the FoF kernels and only the halo properties wait for it.
#include "jfof_internal.cuh"
#include "k_fof.cuh"

using namespace jfof;

namespace {

int ensure_copy_stream(jfof_ctx *ctx) {
    if (ctx->copy_stream) return JFOF_OK;
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return JFOF_ECUDA;
    if (cudaEventCreateWithFlags(&ctx->ev_pos, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_vel, cudaEventDisableTiming) != cudaSuccess)
        return JFOF_ECUDA;
    return JFOF_OK;
}

}  // namespace

extern "C" {

int jfof_fof_host(jfof_ctx *ctx, const float *h_pos, const float *h_vel, int64_t N, float L, float b,
                  int32_t n_axis, uint32_t flags, int32_t min_size, float particle_mass, float *d_pos, float *d_vel,
                  void *ws, size_t ws_bytes, int32_t *label, int32_t *halo_id, int32_t *count, int32_t *halo_start,
                  int32_t *members, int32_t *n_halos, float *mass, float *com, float *vmean, float *sigv) {
    if (!ctx || !h_pos || !d_pos || !ws || !mass || !com) return JFOF_EINVAL;
    if ((h_vel == nullptr) != (d_vel == nullptr)) return JFOF_EINVAL;
    if (h_vel && (!vmean || !sigv)) return JFOF_EINVAL;
    if (!label || !halo_id || !count || !halo_start || !members || !n_halos || min_size < 1) return JFOF_EINVAL;
    int e = check_box(N, L, b);
    if (e) return e;
    int32_t n;
    if ((e = resolve_n(N, L, b, n_axis, &n))) return e;
    size_t need = 0;
    if ((e = jfof_fof_all_bytes(N, n, &need))) return e;
    if (ws_bytes < need) return JFOF_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return JFOF_ECUDA;
    if (h_vel && (e = ensure_copy_stream(ctx))) return e;
    const size_t bytes = sizeof(float) * 3 * size_t(N);
    if (cudaMemcpyAsync(d_pos, h_pos, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) return JFOF_ECUDA;
    if (h_vel) {
        if (cudaEventRecord(ctx->ev_pos, ctx->stream) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_pos, 0) != cudaSuccess ||
            cudaMemcpyAsync(d_vel, h_vel, bytes, cudaMemcpyHostToDevice, ctx->copy_stream) != cudaSuccess ||
            cudaEventRecord(ctx->ev_vel, ctx->copy_stream) != cudaSuccess)
            return JFOF_ECUDA;
    }
    e = jfof_fof(ctx, d_pos, N, L, b, n, flags, min_size, ws, ws_bytes, label, halo_id, count, halo_start, members,
                 n_halos);
    // the context's stream never runs ahead of the velocity upload (waited on
    // even when jfof_fof failed, so the copy stream is never left behind)
    if (h_vel && cudaStreamWaitEvent(ctx->stream, ctx->ev_vel, 0) != cudaSuccess && !e) e = JFOF_ECUDA;
    if (e) return e;
    int64_t H_cap = N / min_size;
    if (H_cap < 1) H_cap = 1;
    return jfof_halo_props(ctx, d_pos, d_vel, N, L, flags, halo_start, members, n_halos, H_cap, particle_mass, mass,
                           com, vmean, sigv);
}

}  // extern "C"
