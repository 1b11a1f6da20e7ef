// k_fof.cuh -- host-side launchers of the FoF kernels (internal).
#pragma once
#include <cmath>

#include "jfof_internal.cuh"

namespace jfof {

// Dense-cell path: sub-cells per cell side (at most), their count, and the
// largest cell it takes (sub-cell offsets are stored as uint16).
constexpr int kSubSide = 9;
constexpr int kSubMax = kSubSide * kSubSide * kSubSide;  // 729
constexpr uint32_t kDenseMaxM = 65535;
// Dense threshold when none is set (kDenseAuto): 160 for boxes of more than
// 2^23 particles, where it measured fastest; 96 below (the boxes of a batch),
// where a box's time is set by its slowest cells and a large medium cell
// takes longer than the dense path for it.
constexpr int kDenseAuto = -1;
inline int default_dense_threshold(int64_t N) { return N > (int64_t(1) << 23) ? 160 : 96; }
constexpr int kDefaultSmallThreshold = 16;
constexpr int kSmallMax = 255;  // small cells hold at most this many particles
// Medium cells (more than S particles, not on the dense path) are listed in
// one array: cells of at most kMedMain particles from its front, larger ones
// from its back.  Up to kMedBig particles their pairs are found through
// adjacency bitmasks and reach sets of 32-bit words.
constexpr int kMedMain = 96;
constexpr int kMedBig = 160;
// dense cells, medium cells, four work counters, small-cell particles, small
// work counter, large medium cells, two work counters
constexpr int kCounters = 12;
// Output-order buckets of the label scatter (at most this many).
constexpr int kTailBuckets = 1024;
// Binning of grids with at most kFewBricks bricks: a counting sort by
// kFewGrid CTAs over contiguous chunks (no global atomics).  The chunk count
// is fixed (two per SM of a GB300); results do not depend on it.
constexpr int kFewBricks = 4096;
constexpr int kFewGrid = 304;

// One IEEE binary32 multiply on the host (b*b for the link threshold).
inline float host_mul(float a, float b) {
    volatile float r = a * b;
    return r;
}

inline int64_t dense_cap(int64_t N) { return N / 256 + 1024; }
inline int64_t medium_cap(int64_t N) { return N + 16; }

// Views into the bin/link workspace.
struct FofBuffers {
    float4 *spos;
    uint32_t *cell_start;
    uint32_t *brick_count;
    uint32_t *brick_start;
    uint32_t *cursor;
    uint32_t *scan_tmp;
    float4 *tmp;           // bin scatter; dense-cell staging; then rootmin
    int *parent;           // [N]
    uint32_t *dense_id;    // [cell table]
    uint32_t *dense_cells; // [D_cap]
    uint32_t *counters;    // [kCounters]: dense cells, medium cells, four work counters,
                           // small-cell particles, small work counter, large medium
                           // cells, their two work counters
    uint32_t *small_slots; // [N] slots of the particles of small cells
    uint16_t *sub_start;   // [D_cap][kSubMax + 1]
    uint16_t *sub_rows;    // [D_cap][kSubSide^2] bit x of row (y, z): sub-cell non-empty
    uint32_t *medium_cells;// [medium_cap] medium cells from the front, large ones from the back
    uint32_t *bucket_fill; // [kTailBuckets] label-scatter bucket cursors
    uint32_t *bin_mat;     // [kFewGrid][bricks] per-CTA brick counts (few-brick grids)
    uint32_t *bin_base;    // [bricks * kFewGrid + 1] their brick-major exclusive scan
};

// Dense-path parameters derived on the host from (N, L, b, n, T), and the
// CTA shape of the list-driven link kernels (a tuning knob; results do not
// depend on it): warps per CTA of medium_local, medium, dense_cells and
// dense_nbr.  Shape 0 = (4, 8, 4, 8), 1 = all 8, 2 = all 4.
constexpr int kCtaShapes = 3;
struct LinkParams {
    int S;          // small cells: at most S particles
    int T;          // dense threshold actually used (0 = dense path off)
    int k;          // sub-cells per cell side
    float inv_fine; // f32(n k / L)
    int64_t D_cap;  // dense cells with a sub-cell table
    int warps[4];   // warps per CTA of the four list-driven link kernels
};

size_t fof_layout(int64_t N, int n, FofBuffers *fb, void *base);

// Host-side argument rules shared by the ABI entry points (api.cu).
bool finite_pos(float x);
int check_box(int64_t N, float L, float b);
int32_t max_cells(float L, float b);
int resolve_n(int64_t N, float L, float b, int32_t n_axis, int32_t *out);
LinkParams make_link_params(int64_t N, float L, float b, int n, int S, int T, int shape = 0);
void launch_bin_cells(const float *pos, int64_t N, float L, int n, bool wrap, const LinkParams &lp,
                      const FofBuffers &fb, const DevStatus &st, cudaStream_t s);
// Union-find over the cell grid (parent[] complete, not yet flattened).
void launch_link_core(const jfof_cells &c, const FofBuffers &fb, const LinkParams &lp, const DevStatus &st,
                      cudaStream_t s);
// Core, then raw labels in original order.
void launch_link(const jfof_cells &c, const FofBuffers &fb, const LinkParams &lp, int32_t *label,
                 const DevStatus &st, cudaStream_t s);

// Groups.
struct GroupBuffers {
    uint32_t *cnt;   // [N]
    uint32_t *hid;   // [N+1]
    uint32_t *cursor;// [H_cap+1]
    uint32_t *scan_tmp;
    uint32_t *seglist;  // segmented-sort list of long halos
    int64_t seglist_words;
    int32_t *hlabel;    // [H_cap] raw label of each halo
};
size_t groups_layout(int64_t N, int64_t H_cap, GroupBuffers *gb, void *base);
void launch_groups(const int32_t *label, int64_t N, int32_t min_size, int64_t H_cap, const GroupBuffers &gb,
                   int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members, int32_t *n_halos,
                   const DevStatus &st, cudaStream_t s);

// After launch_link_core: raw labels only, or labels with the whole of a7
// computed from the forest (same outputs as launch_link + launch_groups).
void launch_tail_labels(const FofBuffers &fb, int64_t N, int32_t *label, cudaStream_t s);
void launch_tail_groups(const FofBuffers &fb, int64_t N, int32_t min_size, int64_t H_cap, const GroupBuffers &gb,
                        int32_t *label, int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members,
                        int32_t *n_halos, cudaStream_t s);

// Properties.
void launch_halo_props(const float *pos, const float *vel, int64_t N, float L, bool wrap, const int32_t *halo_start,
                       const int32_t *members, const int32_t *n_halos, int64_t H_cap, float particle_mass,
                       float *mass, float *com, float *vmean, float *sigv, cudaStream_t s);
void launch_halo_props_backward(const float *vel, const int32_t *halo_id, const int32_t *count, int64_t N,
                                const float *vmean, const float *sigv, const float *g_com, const float *g_vmean,
                                const float *g_sigv, float *g_pos, float *g_vel, cudaStream_t s);

}  // namespace jfof
