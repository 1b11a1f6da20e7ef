// k_props.cu -- a8/a9: halo properties and their frozen-assignment adjoint
// (Sec. 3.1, Eq. 4; Table 1).  Binary32 with compensated (Kahan) sums in a
// fixed order, so results are deterministic run to run.
#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {

// Kahan accumulator: value = s - c.
struct KSum {
    float s, c;
};

__device__ __forceinline__ void kadd(KSum &a, float x) {
    float y = __fsub_rn(x, a.c);
    float t = __fadd_rn(a.s, y);
    a.c = __fsub_rn(__fsub_rn(t, a.s), y);
    a.s = t;
}

// Exact-error merge of two compensated sums (TwoSum on the heads).
__device__ __forceinline__ KSum kmerge(KSum a, KSum b) {
    float s = __fadd_rn(a.s, b.s);
    float bb = __fsub_rn(s, a.s);
    float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(b.s, bb));
    KSum r;
    r.s = s;
    r.c = __fsub_rn(__fadd_rn(a.c, b.c), e);
    return r;
}

__device__ __forceinline__ KSum kwarp(KSum a) {
    for (int o = 16; o > 0; o >>= 1) {
        KSum b;
        b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
        b.c = __shfl_xor_sync(0xffffffffu, a.c, o);
        // lanes l and l^o both compute merge(lower lane, upper lane) so the
        // result is identical in both lanes
        int lane = threadIdx.x & 31;
        a = (lane & o) ? kmerge(b, a) : kmerge(a, b);
    }
    return a;
}

__device__ __forceinline__ float kval(KSum a) { return __fsub_rn(a.s, a.c); }

__device__ __forceinline__ float load_coord(const float *pos, int64_t i, int a, float L, bool wrap) {
    float x = pos[3 * i + a];
    return wrap ? wrap_coord(x, L) : x;
}

// Running (count, mean, sum of squared deviations) of a lane's velocities
// (Welford's update) and the exact pairwise merge of two such summaries
// (Chan, Golub & LeVeque): M2 = M2a + M2b + d^2 na nb / (na + nb) with
// d = mean_b - mean_a.  Every term added to M2 is non-negative, so no large
// terms cancel whatever the velocities are (a cold halo whose first member is
// an outlier included); the mean is a compensated-free running average whose
// rounding enters M2 only at second order.
struct Moments {
    float n, m[3], M2;
};

__device__ __forceinline__ void welford(Moments &a, const float v[3]) {
    a.n = __fadd_rn(a.n, 1.0f);
    const float r = __frcp_rn(a.n);
    float q = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float d = __fsub_rn(v[c], a.m[c]);
        a.m[c] = __fadd_rn(a.m[c], __fmul_rn(d, r));
        q = __fadd_rn(q, __fmul_rn(d, __fsub_rn(v[c], a.m[c])));
    }
    a.M2 = __fadd_rn(a.M2, q);
}

__device__ __forceinline__ Moments chan(const Moments &a, const Moments &b) {
    if (a.n == 0.f) return b;
    if (b.n == 0.f) return a;
    Moments r;
    r.n = __fadd_rn(a.n, b.n);
    const float wb = __fdiv_rn(b.n, r.n);
    float dd = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float d = __fsub_rn(b.m[c], a.m[c]);
        r.m[c] = __fadd_rn(a.m[c], __fmul_rn(d, wb));
        dd = __fadd_rn(dd, __fmul_rn(d, d));
    }
    r.M2 = __fadd_rn(__fadd_rn(a.M2, b.M2), __fmul_rn(dd, __fmul_rn(a.n, wb)));
    return r;
}

// Warp merge in a fixed butterfly order (each pair merges lower lane first,
// so all lanes end with the same summary).
__device__ __forceinline__ Moments chan_warp(Moments a) {
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
        Moments b;
        b.n = __shfl_xor_sync(0xffffffffu, a.n, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) b.m[c] = __shfl_xor_sync(0xffffffffu, a.m[c], o);
        b.M2 = __shfl_xor_sync(0xffffffffu, a.M2, o);
        a = (lane & o) ? chan(b, a) : chan(a, b);
    }
    return a;
}

// One warp per halo (grid-stride over halos), one gather pass over the
// members.  Positions are summed as minimum-image offsets from the halo's
// first member xr (periodic centre of mass) and velocities as offsets from
// that member's velocity vr, both compensated: vmean = vr + S1/m.  The
// dispersion comes from the Welford summaries of each lane's velocities,
// merged across the warp by Chan's formula: sigma^2 = M2 / (3 m), with no
// cancellation.
__global__ void __launch_bounds__(256) halo_props_kernel(const float *__restrict__ pos, const float *__restrict__ vel,
                                                         float L, bool wrap, const int32_t *__restrict__ halo_start,
                                                         const int32_t *__restrict__ members,
                                                         const int32_t *__restrict__ n_halos, float particle_mass,
                                                         float *__restrict__ mass, float *__restrict__ com,
                                                         float *__restrict__ vmean, float *__restrict__ sigv) {
    int H = *n_halos;
    int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    float hL = 0.5f * L;
    for (int64_t h = warp; h < H; h += nwarps) {
        int hs = halo_start[h], he = halo_start[h + 1];
        int m = he - hs;
        float fm = float(m);
        int r = members[hs];  // smallest member: the segment is sorted
        float xr[3], vr[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xr[a] = load_coord(pos, r, a, L, wrap);
            if (vel) vr[a] = vel[3 * int64_t(r) + a];
        }
        KSum sx[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        KSum sv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        Moments mv{0.f, {0.f, 0.f, 0.f}, 0.f};
        constexpr int U = 4;  // members per lane per step: all gathers issue before the sums
        for (int k0 = hs + lane; k0 < he; k0 += 32 * U) {
            int idx[U];
            bool on[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                on[u] = k0 + 32 * u < he;
                idx[u] = on[u] ? members[k0 + 32 * u] : members[k0];
            }
            float pp[U][3], vv[U][3];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    pp[u][a] = load_coord(pos, idx[u], a, L, wrap);
                    vv[u][a] = vel ? vel[3 * int64_t(idx[u]) + a] : 0.f;
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!on[u]) continue;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    kadd(sx[a], min_image(pp[u][a], xr[a], L, hL));
                    if (vel) kadd(sv[a], __fsub_rn(vv[u][a], vr[a]));
                }
                if (vel) welford(mv, vv[u]);
            }
        }
        float vm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float d = __fdiv_rn(kval(kwarp(sx[a])), fm);
            float c = wrap_coord(__fadd_rn(xr[a], d), L);
            if (lane == 0) com[3 * h + a] = c;
            vm[a] = vel ? __fadd_rn(vr[a], __fdiv_rn(kval(kwarp(sv[a])), fm)) : 0.f;
        }
        if (lane == 0) mass[h] = __fmul_rn(particle_mass, fm);
        if (!vel) continue;
        const Moments t = chan_warp(mv);
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) vmean[3 * h + a] = vm[a];
            sigv[h] = __fsqrt_rn(fmaxf(__fdiv_rn(t.M2, __fmul_rn(3.0f, fm)), 0.f));
        }
    }
}

void launch_halo_props(const float *pos, const float *vel, int64_t N, float L, bool wrap, const int32_t *halo_start,
                       const int32_t *members, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                       float *mass, float *com, float *vmean, float *sigv, cudaStream_t s) {
    (void)N;
    {
        JFOF_TRACE("halo_props", s);
        halo_props_kernel<<<grid_for(H_cap * 32, 256, 8), 256, 0, s>>>(pos, vel, L, wrap, halo_start, members, n_halos,
                                                                      particle_mass, mass, com, vmean, sigv);
    }
}

// Adjoint: one thread per particle (streams halo_id, vel, writes g_pos, g_vel).
__global__ void __launch_bounds__(256) halo_props_bwd_kernel(const float *__restrict__ vel,
                                                             const int32_t *__restrict__ halo_id,
                                                             const int32_t *__restrict__ count, int64_t N,
                                                             const float *__restrict__ vmean,
                                                             const float *__restrict__ sigv,
                                                             const float *__restrict__ g_com,
                                                             const float *__restrict__ g_vmean,
                                                             const float *__restrict__ g_sigv,
                                                             float *__restrict__ g_pos, float *__restrict__ g_vel) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        int32_t h = halo_id[i];
        float gp[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
        if (h >= 0) {
            float fn = float(count[h]);
            float coef = 0.f;
            if (g_sigv) {
                float sg = sigv[h];
                if (sg > 0.f) coef = __fdiv_rn(g_sigv[h], __fmul_rn(__fmul_rn(3.0f, fn), sg));
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (g_com) gp[a] = __fdiv_rn(g_com[3 * int64_t(h) + a], fn);
                float v = 0.f;
                if (g_vmean) v = __fdiv_rn(g_vmean[3 * int64_t(h) + a], fn);
                if (coef != 0.f)
                    v = __fadd_rn(v, __fmul_rn(coef, __fsub_rn(vel[3 * i + a], vmean[3 * int64_t(h) + a])));
                gv[a] = v;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (g_pos) g_pos[3 * i + a] = gp[a];
            if (g_vel) g_vel[3 * i + a] = gv[a];
        }
    }
}

void launch_halo_props_backward(const float *vel, const int32_t *halo_id, const int32_t *count, int64_t N,
                                const float *vmean, const float *sigv, const float *g_com, const float *g_vmean,
                                const float *g_sigv, float *g_pos, float *g_vel, cudaStream_t s) {
    {
        JFOF_TRACE("halo_props_bwd", s);
        halo_props_bwd_kernel<<<grid_for(N, 256), 256, 0, s>>>(vel, halo_id, count, N, vmean, sigv, g_com, g_vmean,
                                                              g_sigv, g_pos, g_vel);
    }
}

}  // namespace jfof
