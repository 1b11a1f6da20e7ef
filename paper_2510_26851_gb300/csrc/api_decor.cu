// api_decor.cu -- C ABI of the decorated frozen assignment and the soft
// mass function (Sec. 3.1.1, Eq. 5): argument checks and launches.
#include <cmath>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {
int soft_hist_blocks(int64_t H_cap);
void launch_halo_decoration(const float *pos, float L, bool wrap, const int32_t *halo_start, const int32_t *members,
                            const int32_t *n_halos, int64_t H_cap, const float *com, float *dsig, cudaStream_t s);
void launch_halo_decoration_backward(const float *pos, float L, bool wrap, const int32_t *halo_id,
                                     const int32_t *count, int64_t N, const float *com, const float *dsig,
                                     const float *g_dsig, float *g_pos, cudaStream_t s);
void launch_soft_hist(const int32_t *count, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                      const float *edges, int B, float width, float *partial, float *hist, cudaStream_t s);
void launch_soft_hist_backward(const int32_t *count, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                               const float *dsig, const float *edges, int B, float width, float kappa,
                               const float *g_hist, float *g_dsig, cudaStream_t s);
}  // namespace jfof

using namespace jfof;

namespace {
int launched() { return cudaGetLastError() == cudaSuccess ? JFOF_OK : JFOF_ECUDA; }
constexpr int32_t kMaxBins = 4096;
}  // namespace

extern "C" {

int jfof_halo_decoration(jfof_ctx *ctx, const float *pos, int64_t N, float L, uint32_t flags,
                         const int32_t *halo_start, const int32_t *members, const int32_t *n_halos, int64_t H_cap,
                         const float *com, float *dsig) {
    if (!ctx || !pos || !halo_start || !members || !n_halos || !com || !dsig) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX) || H_cap < 1 || !finite_pos(L)) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_halo_decoration(pos, L, (flags & JFOF_WRAP) != 0, halo_start, members, n_halos, H_cap, com, dsig,
                           ctx->stream);
    return launched();
}

int jfof_halo_decoration_backward(jfof_ctx *ctx, const float *pos, const int32_t *halo_id, const int32_t *count,
                                  int64_t N, float L, uint32_t flags, const float *com, const float *dsig,
                                  const float *g_dsig, float *g_pos) {
    if (!ctx || !pos || !halo_id || !count || !com || !dsig || !g_dsig || !g_pos) return JFOF_EINVAL;
    if (N < 1 || N > int64_t(INT32_MAX) || !finite_pos(L)) return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_halo_decoration_backward(pos, L, (flags & JFOF_WRAP) != 0, halo_id, count, N, com, dsig, g_dsig, g_pos,
                                    ctx->stream);
    return launched();
}

int jfof_soft_hmf_bytes(int64_t H_cap, int32_t B, size_t *bytes) {
    if (!bytes || H_cap < 1 || B < 1 || B > kMaxBins) return JFOF_EINVAL;
    *bytes = sizeof(float) * size_t(soft_hist_blocks(H_cap)) * size_t(B);
    return JFOF_OK;
}

int jfof_soft_hmf(jfof_ctx *ctx, const int32_t *count, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                  const float *edges, int32_t B, float width, void *ws, size_t ws_bytes, float *hist) {
    if (!ctx || !count || !n_halos || !edges || !ws || !hist) return JFOF_EINVAL;
    if (H_cap < 1 || B < 1 || B > kMaxBins || !finite_pos(width) || !finite_pos(particle_mass)) return JFOF_EINVAL;
    size_t need = 0;
    jfof_soft_hmf_bytes(H_cap, B, &need);
    if (ws_bytes < need) return JFOF_ENOMEM;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_soft_hist(count, n_halos, H_cap, particle_mass, edges, B, width, reinterpret_cast<float *>(ws), hist,
                     ctx->stream);
    return launched();
}

int jfof_soft_hmf_backward(jfof_ctx *ctx, const int32_t *count, const int32_t *n_halos, int64_t H_cap,
                           float particle_mass, const float *dsig, const float *edges, int32_t B, float width,
                           float kappa, const float *g_hist, float *g_dsig) {
    if (!ctx || !count || !n_halos || !dsig || !edges || !g_hist || !g_dsig) return JFOF_EINVAL;
    if (H_cap < 1 || B < 1 || B > kMaxBins || !finite_pos(width) || !finite_pos(particle_mass) ||
        !std::isfinite(kappa))
        return JFOF_EINVAL;
    cudaSetDevice(ctx->device);
    CtxScope scope(ctx);
    launch_soft_hist_backward(count, n_halos, H_cap, particle_mass, dsig, edges, B, width, kappa, g_hist, g_dsig,
                              ctx->stream);
    return launched();
}

}  // extern "C"
