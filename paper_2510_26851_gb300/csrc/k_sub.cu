// k_sub.cu -- sub-halos (Sec. 2.1.1, Eq. 3): a second Friends-of-Friends pass
// inside each halo in phase space.  Members i, j of one halo are friends when
//   |x_i - x_j|^2 / sigma_x + |v_i - v_j|^2 / sigma_v <= 1
// (minimum-image position difference), evaluated in binary32 in a fixed
// order with no fused operations,
//   dxx = (dx*dx + dy*dy) + dz*dz,  dvv = (du*du + dv*dv) + dw*dw,
//   link iff dxx * inv_sx + dvv * inv_sv <= 1,
// so that the groups are bit-identical to a plain evaluation of the same
// expression.  The halo's members (CSR, ascending index) are first gathered
// into member order; one warp per halo then tests every pair once (rows r and
// m-1-r per lane, so every lane has m-1 pairs per step) and unites linked
// pairs in a forest over member slots whose root is the smallest slot, i.e.
// the smallest member index.
#include <cmath>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {

namespace {

__device__ __forceinline__ float phase_d2(float4 xi, float4 xj, float4 vi, float4 vj, float L, float hL,
                                          float inv_sx, float inv_sv) {
    const float dx = min_image(xj.x, xi.x, L, hL), dy = min_image(xj.y, xi.y, L, hL),
                dz = min_image(xj.z, xi.z, L, hL);
    const float du = __fsub_rn(vj.x, vi.x), dv = __fsub_rn(vj.y, vi.y), dw = __fsub_rn(vj.z, vi.z);
    const float dxx = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const float dvv = __fadd_rn(__fadd_rn(__fmul_rn(du, du), __fmul_rn(dv, dv)), __fmul_rn(dw, dw));
    return __fadd_rn(__fmul_rn(dxx, inv_sx), __fmul_rn(dvv, inv_sv));
}

}  // namespace

// Members' positions and velocities in member order; every slot its own root.
__global__ void __launch_bounds__(256) sub_gather_kernel(const float *__restrict__ pos, const float *__restrict__ vel,
                                                         float L, bool wrap, const int32_t *__restrict__ halo_start,
                                                         const int32_t *__restrict__ members,
                                                         const int32_t *__restrict__ n_halos, int64_t N,
                                                         float4 *__restrict__ xs, float4 *__restrict__ vs,
                                                         int *__restrict__ par) {
    const int64_t M = halo_start[*n_halos];
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < M && k < N;
         k += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = members[k];
        float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (wrap) {
            x = wrap_coord(x, L);
            y = wrap_coord(y, L);
            z = wrap_coord(z, L);
        }
        xs[k] = make_float4(x, y, z, 0.f);
        vs[k] = make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.f);
        par[k] = int(k);
    }
}

// One warp per halo: every pair of members once; a linked pair is united.
__global__ void __launch_bounds__(256) sub_link_kernel(const int32_t *__restrict__ halo_start,
                                                       const int32_t *__restrict__ n_halos,
                                                       const float4 *__restrict__ xs, const float4 *__restrict__ vs,
                                                       float L, float inv_sx, float inv_sv, int *par, DevStatus st) {
    const int H = *n_halos;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const float hL = 0.5f * L;
    for (int64_t h = warp; h < H; h += nwarps) {
        const int hs = halo_start[h], m = halo_start[h + 1] - hs;
        const int half = (m + 1) / 2;
        for (int r = lane; r < half; r += 32) {
            // row r (pairs with r+1 .. m-1) and its mirror row m-1-r
            for (int pass = 0; pass < 2; ++pass) {
                const int a = pass == 0 ? r : m - 1 - r;
                if (pass == 1 && a == r) break;
                const float4 xa = xs[hs + a], va = vs[hs + a];
                for (int c = a + 1; c < m; ++c)
                    if (phase_d2(xa, xs[hs + c], va, vs[hs + c], L, hL, inv_sx, inv_sv) <= 1.0f)
                        uf_unite(par, hs + a, hs + c, st);
            }
        }
    }
}

// Sub-labels: every particle its own group, then members get the smallest
// member index of their phase-space group.
__global__ void __launch_bounds__(256) sub_init_kernel(int32_t *__restrict__ sub_label, int64_t N) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
        sub_label[i] = int32_t(i);
}

__global__ void __launch_bounds__(256) sub_label_kernel(const int32_t *__restrict__ halo_start,
                                                        const int32_t *__restrict__ members,
                                                        const int32_t *__restrict__ n_halos, int64_t N,
                                                        const int *__restrict__ par,
                                                        int32_t *__restrict__ sub_label) {
    const int64_t M = halo_start[*n_halos];
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < M && k < N;
         k += int64_t(gridDim.x) * blockDim.x)
        sub_label[members[k]] = members[uf_find_ro(par, int(k))];
}

size_t subhalo_layout(int64_t N, float4 **xs, float4 **vs, int **par, void *base) {
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    float4 *a = reinterpret_cast<float4 *>(take(sizeof(float4) * size_t(N)));
    float4 *b = reinterpret_cast<float4 *>(take(sizeof(float4) * size_t(N)));
    int *c = reinterpret_cast<int *>(take(sizeof(int) * size_t(N)));
    if (xs) *xs = a;
    if (vs) *vs = b;
    if (par) *par = c;
    return off;
}

void launch_subhalos(const float *pos, const float *vel, int64_t N, float L, bool wrap, const int32_t *halo_start,
                     const int32_t *members, const int32_t *n_halos, int64_t H_cap, float inv_sx, float inv_sv,
                     void *ws, int32_t *sub_label, const DevStatus &st, cudaStream_t s) {
    float4 *xs, *vs;
    int *par;
    subhalo_layout(N, &xs, &vs, &par, ws);
    {
        JFOF_TRACE("sub_gather", s);
        sub_gather_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, vel, L, wrap, halo_start, members, n_halos, N, xs,
                                                          vs, par);
    }
    {
        JFOF_TRACE("sub_link", s);
        sub_link_kernel<<<grid_for(H_cap * 32, 256, 8), 256, 0, s>>>(halo_start, n_halos, xs, vs, L, inv_sx, inv_sv,
                                                                    par, st);
    }
    {
        JFOF_TRACE("sub_labels", s);
        sub_init_kernel<<<grid_for(N, 256), 256, 0, s>>>(sub_label, N);
        sub_label_kernel<<<grid_for(N, 256), 256, 0, s>>>(halo_start, members, n_halos, N, par, sub_label);
    }
}

}  // namespace jfof
