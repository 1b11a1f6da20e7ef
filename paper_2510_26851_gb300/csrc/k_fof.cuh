// k_fof.cuh -- host-side launchers of the FoF kernels (internal).
#pragma once
#include "jfof_internal.cuh"

namespace jfof {

// One IEEE binary32 multiply on the host (b*b for the link threshold).
inline float host_mul(float a, float b) {
    volatile float r = a * b;
    return r;
}

// Views into the bin/link workspace.
struct FofBuffers {
    float4 *spos;
    uint32_t *cell_start;
    uint32_t *brick_count;
    uint32_t *brick_start;
    uint32_t *cursor;
    uint32_t *scan_tmp;
    float4 *tmp;  // also the link scratch (parent, rootmin)
};

size_t fof_layout(int64_t N, int n, FofBuffers *fb, void *base);
void launch_bin_cells(const float *pos, int64_t N, float L, int n, bool wrap, const FofBuffers &fb,
                      const DevStatus &st, cudaStream_t s);
void launch_link(const jfof_cells &c, int32_t *label, const DevStatus &st, cudaStream_t s);

// Groups.
struct GroupBuffers {
    uint32_t *cnt;   // [N]
    uint32_t *hid;   // [N+1]
    uint32_t *cursor;// [H_cap+1]
    uint32_t *scan_tmp;
};
size_t groups_layout(int64_t N, int64_t H_cap, GroupBuffers *gb, void *base);
void launch_groups(const int32_t *label, int64_t N, int32_t min_size, int64_t H_cap, const GroupBuffers &gb,
                   int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members, int32_t *n_halos,
                   const DevStatus &st, cudaStream_t s);

// Properties.
void launch_halo_props(const float *pos, const float *vel, int64_t N, float L, bool wrap, const int32_t *halo_start,
                       const int32_t *members, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                       float *mass, float *com, float *vmean, float *sigv, cudaStream_t s);
void launch_halo_props_backward(const float *vel, const int32_t *halo_id, const int32_t *count, int64_t N,
                                const float *vmean, const float *sigv, const float *g_com, const float *g_vmean,
                                const float *g_sigv, float *g_pos, float *g_vel, cudaStream_t s);

}  // namespace jfof
