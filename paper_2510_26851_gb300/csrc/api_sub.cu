// api_sub.cu -- C ABI of the phase-space sub-halo pass (Sec. 2.1.1, Eq. 3).
#include <cmath>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {
size_t subhalo_layout(int64_t N, float4 **xs, float4 **vs, int **par, void *base);
void launch_subhalos(const float *pos, const float *vel, int64_t N, float L, bool wrap, const int32_t *halo_start,
                     const int32_t *members, const int32_t *n_halos, int64_t H_cap, float inv_sx, float inv_sv,
                     void *ws, int32_t *sub_label, const DevStatus &st, cudaStream_t s);
}  // namespace jfof

using namespace jfof;

namespace {

// f32(1/sigma) from double; an infinite scale switches its term off.
bool inverse_scale(float sigma, float *inv) {
    if (std::isinf(sigma) && sigma > 0.0f) {
        *inv = 0.0f;
        return true;
    }
    if (!finite_pos(sigma)) return false;
    *inv = float(1.0 / double(sigma));
    return true;
}

}  // namespace

extern "C" {

int jfof_subhalos_bytes(int64_t N, size_t *bytes) {
    if (!bytes || N < 1 || N > int64_t(INT32_MAX)) return JFOF_EINVAL;
    *bytes = subhalo_layout(N, nullptr, nullptr, nullptr, nullptr);
    return JFOF_OK;
}

int jfof_subhalos(jfof_ctx *ctx, const float *pos, const float *vel, int64_t N, float L, uint32_t flags,
                  const int32_t *halo_start, const int32_t *members, const int32_t *n_halos, int64_t H_cap,
                  float sigma_x, float sigma_v, void *ws, size_t ws_bytes, int32_t *sub_label) {
    if (!ctx || !pos || !vel || !halo_start || !members || !n_halos || !ws || !sub_label) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX) || H_cap < 1 || !finite_pos(L)) return JFOF_EINVAL;
    float inv_sx, inv_sv;
    if (!inverse_scale(sigma_x, &inv_sx) || !inverse_scale(sigma_v, &inv_sv)) return JFOF_EINVAL;
    if (ws_bytes < subhalo_layout(N, nullptr, nullptr, nullptr, nullptr)) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_subhalos(pos, vel, N, L, (flags & JFOF_WRAP) != 0, halo_start, members, n_halos, H_cap, inv_sx, inv_sv,
                    ws, sub_label, ctx->dev(), ctx->stream);
    return cudaGetLastError() == cudaSuccess ? JFOF_OK : JFOF_ECUDA;
}

}  // extern "C"
