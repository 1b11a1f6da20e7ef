// k_decor.cu -- the decorated frozen assignment of Sec. 3.1.1 (Eq. 5): a halo
// "decoration" that is an analytic function of the member positions -- the
// particle standard deviation about the halo centre,
//   D_h = sqrt( sum_i |mi(x_i - X_h)|^2 / (3 n_h) ),
// used as a differentiable proxy for the halo mass -- its frozen-assignment
// adjoint, and a soft (logistic) histogram of the halo log-masses with its
// vector-Jacobian product, through which the mass-function gradient reaches
// the decoration and the positions.  Binary32 with compensated sums in a
// fixed order; every result is deterministic run to run.
#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {

namespace {

struct Comp {
    float s, c;
};

__device__ __forceinline__ void cadd(Comp &a, float x) {
    float y = __fsub_rn(x, a.c);
    float t = __fadd_rn(a.s, y);
    a.c = __fsub_rn(__fsub_rn(t, a.s), y);
    a.s = t;
}

// Warp sum of compensated partials in a fixed butterfly order (both lanes of
// a pair merge lower-then-upper, so every lane ends with the same value).
__device__ __forceinline__ float cwarp(Comp a) {
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
        Comp b{__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o)};
        const Comp lo = (lane & o) ? b : a, hi = (lane & o) ? a : b;
        const float s = __fadd_rn(lo.s, hi.s);
        const float bb = __fsub_rn(s, lo.s);
        const float e = __fadd_rn(__fsub_rn(lo.s, __fsub_rn(s, bb)), __fsub_rn(hi.s, bb));
        a.s = s;
        a.c = __fsub_rn(__fadd_rn(lo.c, hi.c), e);
    }
    return __fsub_rn(a.s, a.c);
}

__device__ __forceinline__ float coord(const float *pos, int64_t i, int a, float L, bool wrap) {
    const float x = pos[3 * i + a];
    return wrap ? wrap_coord(x, L) : x;
}

__device__ __forceinline__ float logistic(float t) { return __frcp_rn(__fadd_rn(1.0f, expf(-t))); }

// log-mass of a halo of n particles
__device__ __forceinline__ float log_mass(float particle_mass, int32_t n) {
    return logf(__fmul_rn(particle_mass, float(n)));
}

}  // namespace

// One warp per halo (grid-stride over halos): deviations from the halo's
// centre of mass (minimum image), squared and summed over the members.
__global__ void __launch_bounds__(256) halo_decoration_kernel(const float *__restrict__ pos, float L, bool wrap,
                                                              const int32_t *__restrict__ halo_start,
                                                              const int32_t *__restrict__ members,
                                                              const int32_t *__restrict__ n_halos,
                                                              const float *__restrict__ com,
                                                              float *__restrict__ dsig) {
    const int H = *n_halos;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const float hL = 0.5f * L;
    for (int64_t h = warp; h < H; h += nwarps) {
        const int hs = halo_start[h], he = halo_start[h + 1];
        const float X[3] = {com[3 * h], com[3 * h + 1], com[3 * h + 2]};
        Comp s2{0.f, 0.f};
        for (int k = hs + lane; k < he; k += 32) {
            const int i = members[k];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float d = min_image(coord(pos, i, a, L, wrap), X[a], L, hL);
                cadd(s2, __fmul_rn(d, d));
            }
        }
        const float v = __fdiv_rn(cwarp(s2), __fmul_rn(3.0f, float(he - hs)));
        if (lane == 0) dsig[h] = __fsqrt_rn(fmaxf(v, 0.f));
    }
}

// Adjoint, one thread per particle: g_x_i = g_D[h] * mi(x_i - X_h) / (3 n_h D_h)
// (the deviations sum to zero, so the centre's own dependence drops out).
__global__ void __launch_bounds__(256) halo_decoration_bwd_kernel(const float *__restrict__ pos, float L, bool wrap,
                                                                  const int32_t *__restrict__ halo_id,
                                                                  const int32_t *__restrict__ count, int64_t N,
                                                                  const float *__restrict__ com,
                                                                  const float *__restrict__ dsig,
                                                                  const float *__restrict__ g_dsig,
                                                                  float *__restrict__ g_pos) {
    const float hL = 0.5f * L;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t h = halo_id[i];
        float g[3] = {0.f, 0.f, 0.f};
        if (h >= 0 && dsig[h] > 0.f) {
            const float c = __fdiv_rn(g_dsig[h], __fmul_rn(__fmul_rn(3.0f, float(count[h])), dsig[h]));
#pragma unroll
            for (int a = 0; a < 3; ++a)
                g[a] = __fmul_rn(c, min_image(coord(pos, i, a, L, wrap), com[3 * int64_t(h) + a], L, hL));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) g_pos[3 * i + a] = g[a];
    }
}

// Soft histogram, pass 1: block b sums its contiguous chunk of halos into
// partial[b][k] for every bin k (warp w takes bins w, w + 8, ...).
constexpr int kHistThreads = 256;

__global__ void __launch_bounds__(kHistThreads) soft_hist_partial_kernel(const int32_t *__restrict__ count,
                                                                        const int32_t *__restrict__ n_halos,
                                                                        float particle_mass,
                                                                        const float *__restrict__ edges, int B,
                                                                        float inv_w, float *__restrict__ partial) {
    const int64_t H = *n_halos;
    const int64_t chunk = (H + gridDim.x - 1) / gridDim.x;
    const int64_t lo = int64_t(blockIdx.x) * chunk, hi = lo + chunk < H ? lo + chunk : H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < B; k += kHistThreads / 32) {
        const float e0 = edges[k], e1 = edges[k + 1];
        Comp s{0.f, 0.f};
        for (int64_t h = lo + lane; h < hi; h += 32) {
            const float ell = log_mass(particle_mass, count[h]);
            cadd(s, __fsub_rn(logistic(__fmul_rn(__fsub_rn(ell, e0), inv_w)),
                              logistic(__fmul_rn(__fsub_rn(ell, e1), inv_w))));
        }
        const float v = cwarp(s);
        if (lane == 0) partial[int64_t(blockIdx.x) * B + k] = v;
    }
}

// Pass 2: hist[k] = sum over blocks of partial[b][k], in block order.
__global__ void soft_hist_reduce_kernel(const float *__restrict__ partial, int nblk, int B, float *__restrict__ hist) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < B; k += gridDim.x * blockDim.x) {
        Comp s{0.f, 0.f};
        for (int b = 0; b < nblk; ++b) cadd(s, partial[int64_t(b) * B + k]);
        hist[k] = __fsub_rn(s.s, s.c);
    }
}

// VJP, one thread per halo: g_ell = sum_k g_k (S'(a_k) - S'(a_{k+1})) / w with
// a_k = (ell - e_k)/w and S' = S (1 - S); the decorated log-mass moves with
// -kappa log D, so g_D = -kappa g_ell / D (0 when D = 0).
__global__ void __launch_bounds__(256) soft_hist_bwd_kernel(const int32_t *__restrict__ count,
                                                            const int32_t *__restrict__ n_halos, float particle_mass,
                                                            const float *__restrict__ dsig,
                                                            const float *__restrict__ edges, int B, float inv_w,
                                                            float kappa, const float *__restrict__ g_hist,
                                                            float *__restrict__ g_dsig) {
    const int64_t H = *n_halos;
    for (int64_t h = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; h < H; h += int64_t(gridDim.x) * blockDim.x) {
        const float ell = log_mass(particle_mass, count[h]);
        float sp_prev;
        {
            const float s = logistic(__fmul_rn(__fsub_rn(ell, edges[0]), inv_w));
            sp_prev = __fmul_rn(s, __fsub_rn(1.0f, s));
        }
        Comp acc{0.f, 0.f};
        for (int k = 0; k < B; ++k) {
            const float s = logistic(__fmul_rn(__fsub_rn(ell, edges[k + 1]), inv_w));
            const float sp = __fmul_rn(s, __fsub_rn(1.0f, s));
            cadd(acc, __fmul_rn(g_hist[k], __fsub_rn(sp_prev, sp)));
            sp_prev = sp;
        }
        const float g_ell = __fmul_rn(__fsub_rn(acc.s, acc.c), inv_w);
        const float D = dsig[h];
        g_dsig[h] = D > 0.f ? __fdiv_rn(__fmul_rn(-kappa, g_ell), D) : 0.f;
    }
}

int soft_hist_blocks(int64_t H_cap) {
    int64_t b = (H_cap + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return int(b);
}

void launch_halo_decoration(const float *pos, float L, bool wrap, const int32_t *halo_start, const int32_t *members,
                            const int32_t *n_halos, int64_t H_cap, const float *com, float *dsig, cudaStream_t s) {
    JFOF_TRACE("halo_decoration", s);
    halo_decoration_kernel<<<grid_for(H_cap * 32, 256, 8), 256, 0, s>>>(pos, L, wrap, halo_start, members, n_halos,
                                                                       com, dsig);
}

void launch_halo_decoration_backward(const float *pos, float L, bool wrap, const int32_t *halo_id,
                                     const int32_t *count, int64_t N, const float *com, const float *dsig,
                                     const float *g_dsig, float *g_pos, cudaStream_t s) {
    JFOF_TRACE("halo_decoration_bwd", s);
    halo_decoration_bwd_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, L, wrap, halo_id, count, N, com, dsig, g_dsig,
                                                               g_pos);
}

void launch_soft_hist(const int32_t *count, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                      const float *edges, int B, float width, float *partial, float *hist, cudaStream_t s) {
    const int nblk = soft_hist_blocks(H_cap);
    JFOF_TRACE("soft_hist", s);
    soft_hist_partial_kernel<<<nblk, kHistThreads, 0, s>>>(count, n_halos, particle_mass, edges, B, 1.0f / width,
                                                           partial);
    soft_hist_reduce_kernel<<<(B + 127) / 128, 128, 0, s>>>(partial, nblk, B, hist);
}

void launch_soft_hist_backward(const int32_t *count, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                               const float *dsig, const float *edges, int B, float width, float kappa,
                               const float *g_hist, float *g_dsig, cudaStream_t s) {
    JFOF_TRACE("soft_hist_bwd", s);
    soft_hist_bwd_kernel<<<grid_for(H_cap, 256), 256, 0, s>>>(count, n_halos, particle_mass, dsig, edges, B,
                                                             1.0f / width, kappa, g_hist, g_dsig);
}

}  // namespace jfof
