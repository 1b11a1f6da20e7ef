// k_bin.cu -- a1-a3 of the hot path on sm_103a: wrap and range check,
// binning by brick (16^3 cells) and the in-brick counting sort by cell, which
// writes the particles in cell order (spos) and the brick-major cell table.
//
// Two ways to group particles by brick, chosen by the brick count:
//  * at most kFewBricks bricks: one counting sort over CTA-owned chunks with a
//    shared-memory histogram of all bricks;
//  * more: a histogram of bricks in L2, its scan, and one atomic cursor per
//    brick (the cursors and partially written lines stay in L2).
// The order of particles inside a cell is not part of any output (labels,
// groups and properties are defined on original indices).
#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {

// ---------------------------------------------------------------------------
// Pass 1 (grids of more than kFewBricks bricks): wrap/check, brick histogram
// (L2-resident counters).
struct BinGeom {
    float L, inv_cell;
    int n, nb;
    bool wrap;
};

__device__ __forceinline__ void load_particle(const float *__restrict__ pos, int64_t i, const BinGeom &g,
                                              const DevStatus &st, float &x, float &y, float &z) {
    x = pos[3 * i + 0];
    y = pos[3 * i + 1];
    z = pos[3 * i + 2];
    if (g.wrap) {
        x = wrap_coord(x, g.L);
        y = wrap_coord(y, g.L);
        z = wrap_coord(z, g.L);
    }
    if (!(x >= 0.0f && x < g.L && y >= 0.0f && y < g.L && z >= 0.0f && z < g.L)) latch(st, JFOF_ERANGE);
}

__global__ void __launch_bounds__(256) bin_count_kernel(const float *__restrict__ pos, int64_t N, BinGeom g,
                                                        uint32_t *__restrict__ brick_count, DevStatus st) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        float x, y, z;
        load_particle(pos, i, g, st, x, y, z);
        int ix = cell_coord(x, g.inv_cell, g.n), iy = cell_coord(y, g.inv_cell, g.n), iz = cell_coord(z, g.inv_cell, g.n);
        uint64_t brick = uint64_t(ix >> 4) + uint64_t(g.nb) * (uint64_t(iy >> 4) + uint64_t(g.nb) * uint64_t(iz >> 4));
        atomicAdd(&brick_count[brick], 1u);
    }
}

// Pass 2: scatter each particle to its brick's segment of tmp (the brick
// cursors and partially written lines stay in L2, which combines the writes).
// Four particles per thread per step, so four cursor atomics are in flight
// before the first result is needed.
constexpr int kScatterItems = 4;

__global__ void __launch_bounds__(256) bin_scatter_kernel(const float *__restrict__ pos, int64_t N, BinGeom g,
                                                          uint32_t *__restrict__ cursor, float4 *__restrict__ tmp,
                                                          DevStatus st) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < N; i0 += stride * kScatterItems) {
        float x[kScatterItems], y[kScatterItems], z[kScatterItems];
        uint32_t slot[kScatterItems];
#pragma unroll
        for (int u = 0; u < kScatterItems; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < N) load_particle(pos, i, g, st, x[u], y[u], z[u]);
        }
#pragma unroll
        for (int u = 0; u < kScatterItems; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= N) continue;
            int ix = cell_coord(x[u], g.inv_cell, g.n), iy = cell_coord(y[u], g.inv_cell, g.n),
                iz = cell_coord(z[u], g.inv_cell, g.n);
            uint64_t brick = uint64_t(ix >> 4) + uint64_t(g.nb) * (uint64_t(iy >> 4) + uint64_t(g.nb) * uint64_t(iz >> 4));
            slot[u] = atomicAdd(&cursor[brick], 1u);
        }
#pragma unroll
        for (int u = 0; u < kScatterItems; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < N) tmp[slot[u]] = make_float4(x[u], y[u], z[u], __int_as_float(int(i)));
        }
    }
}

// Passes 1-2 for grids of at most kFewBricks bricks (small boxes), where a
// few hundred brick counters would each take thousands of atomics: a plain
// two-pass counting sort instead.  Each of the kFewGrid CTAs owns a
// contiguous chunk of particles and writes its per-brick counts (one row of
// mat); a scan of mat in brick-major order gives every (brick, CTA) pair the
// start of its run (and every brick its start, at stride kFewGrid); the
// scatter then ranks particles inside the CTA's runs with shared counters.
constexpr int kFewThreads = 256;

__device__ __forceinline__ uint32_t brick_of(float x, float y, float z, const BinGeom &g) {
    int ix = cell_coord(x, g.inv_cell, g.n), iy = cell_coord(y, g.inv_cell, g.n), iz = cell_coord(z, g.inv_cell, g.n);
    return uint32_t(ix >> 4) + uint32_t(g.nb) * (uint32_t(iy >> 4) + uint32_t(g.nb) * uint32_t(iz >> 4));
}

__global__ void __launch_bounds__(kFewThreads) bin_count_few_kernel(const float *__restrict__ pos, int64_t N,
                                                                    BinGeom g, int n_bricks, int64_t chunk,
                                                                    uint32_t *__restrict__ mat, DevStatus st) {
    __shared__ uint32_t hist[kFewBricks];
    for (int k = threadIdx.x; k < n_bricks; k += kFewThreads) hist[k] = 0u;
    __syncthreads();
    const int64_t lo = int64_t(blockIdx.x) * chunk, hi = lo + chunk < N ? lo + chunk : N;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kFewThreads) {
        float x, y, z;
        load_particle(pos, i, g, st, x, y, z);
        atomicAdd(&hist[brick_of(x, y, z, g)], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_bricks; k += kFewThreads) mat[int64_t(blockIdx.x) * n_bricks + k] = hist[k];
}

// mat read in brick-major order: element (brick k, CTA c) at index k*G + c.
struct BrickMajor {
    const uint32_t *mat;
    int64_t nb;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const {
        return mat[(i % kFewGrid) * nb + i / kFewGrid];
    }
};

__global__ void __launch_bounds__(kFewThreads) bin_scatter_few_kernel(const float *__restrict__ pos, int64_t N,
                                                                      BinGeom g, int n_bricks, int64_t chunk,
                                                                      const uint32_t *__restrict__ base,
                                                                      float4 *__restrict__ tmp, DevStatus st) {
    __shared__ uint32_t cur[kFewBricks];
    for (int k = threadIdx.x; k < n_bricks; k += kFewThreads) cur[k] = base[int64_t(k) * kFewGrid + blockIdx.x];
    __syncthreads();
    const int64_t lo = int64_t(blockIdx.x) * chunk, hi = lo + chunk < N ? lo + chunk : N;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kFewThreads) {
        float x, y, z;
        load_particle(pos, i, g, st, x, y, z);
        uint32_t slot = atomicAdd(&cur[brick_of(x, y, z, g)], 1u);
        tmp[slot] = make_float4(x, y, z, __int_as_float(int(i)));
    }
}

// Pass 3: one CTA per brick (persistent loop): shared-memory counting sort of
// the brick's particles by local cell; writes the brick's 4096 cell starts and
// registers every cell with more than S particles in the medium or the dense
// work list.
constexpr int kSortThreads = 512;
constexpr int kSortUnroll = 2;
constexpr int kSmallStage = 4096;  // small-cell slots of a brick staged in shared memory (at most)

// Cell of a particle inside its brick (0..4095).
__device__ __forceinline__ uint32_t local_cell(float4 q, const BinGeom &g) {
    const int ix = cell_coord(q.x, g.inv_cell, g.n), iy = cell_coord(q.y, g.inv_cell, g.n),
              iz = cell_coord(q.z, g.inv_cell, g.n);
    return uint32_t(ix & 15) + 16u * (uint32_t(iy & 15) + 16u * uint32_t(iz & 15));
}

struct ClassReg {
    int S, T;                 // small: m <= S; dense: T < m <= kDenseMaxM (T = 0: none)
    uint32_t *dense_id;       // [cell table]
    uint32_t *dense_cells;    // [D_cap]
    uint32_t *ndense;         // counter
    int64_t D_cap;
    uint32_t *medium_cells;   // [M_cap]
    uint32_t *nmedium;        // counter
    uint32_t *nlarge;         // counter of medium cells of more than kMedMain particles
    int64_t M_cap;
    uint32_t *small_slots;    // [N] slots of the particles of small cells (null: no list)
    uint32_t *nsmall;         // counter
};

__global__ void __launch_bounds__(kSortThreads) brick_sort_kernel(const float4 *__restrict__ tmp,
                                                                  const uint32_t *__restrict__ brick_start,
                                                                  int64_t bstride, int64_t n_bricks, BinGeom g,
                                                                  float4 *__restrict__ spos,
                                                                  uint32_t *__restrict__ cell_start, ClassReg cr) {
    __shared__ uint32_t hist[kBrickCells];
    __shared__ uint32_t stage[kSmallStage];  // the brick's small-cell slots, in order
    __shared__ uint32_t warps[kSortThreads / 32];
    __shared__ uint32_t small_base;
    constexpr int per = kBrickCells / kSortThreads;  // 8
    for (int64_t brick = blockIdx.x; brick < n_bricks; brick += gridDim.x) {
        uint32_t bs = brick_start[brick * bstride], be = brick_start[(brick + 1) * bstride];
        for (int k = threadIdx.x; k < kBrickCells; k += kSortThreads) hist[k] = 0;
        __syncthreads();
        // kSortUnroll loads in flight per thread before their counts
        for (uint32_t e0 = bs + threadIdx.x; e0 < be; e0 += kSortUnroll * kSortThreads) {
            float4 q[kSortUnroll];
#pragma unroll
            for (int u = 0; u < kSortUnroll; ++u) {
                const uint32_t e = e0 + u * kSortThreads;
                if (e < be) q[u] = tmp[e];
            }
#pragma unroll
            for (int u = 0; u < kSortUnroll; ++u)
                if (e0 + u * kSortThreads < be) atomicAdd(&hist[local_cell(q[u], g)], 1u);
        }
        __syncthreads();
        uint32_t v[per];
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            v[k] = hist[threadIdx.x * per + k];
            s += v[k];
        }
        uint32_t total;
        uint32_t pre = block_exclusive_scan(s, warps, &total);
        uint64_t tbase = uint64_t(brick) * kBrickCells;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            uint64_t gidx = tbase + threadIdx.x * per + k;
            hist[threadIdx.x * per + k] = pre;
            cell_start[gidx] = bs + pre;
            pre += v[k];
            if (v[k] > uint32_t(cr.S)) {
                bool dense = false;
                if (cr.T > 0 && v[k] > uint32_t(cr.T) && v[k] <= kDenseMaxM) {
                    uint32_t id = atomicAdd(cr.ndense, 1u);
                    cr.dense_id[gidx] = id;
                    if (int64_t(id) < cr.D_cap) {
                        cr.dense_cells[id] = uint32_t(gidx);
                        dense = true;
                    }
                }
                if (!dense) {
                    // medium cells from the front of the array, large ones from
                    // its back (together at most one per non-empty cell < M_cap)
                    if (v[k] <= uint32_t(kMedMain)) {
                        uint32_t id = atomicAdd(cr.nmedium, 1u);
                        if (int64_t(id) < cr.M_cap) cr.medium_cells[id] = uint32_t(gidx);
                    } else {
                        uint32_t id = atomicAdd(cr.nlarge, 1u);
                        if (int64_t(id) < cr.M_cap) cr.medium_cells[cr.M_cap - 1 - int64_t(id)] = uint32_t(gidx);
                    }
                }
            }
        }
        if (cr.small_slots) {
            // slots of the small cells' particles, appended in cell order
            uint32_t ns = 0;
#pragma unroll
            for (int k = 0; k < per; ++k)
                if (v[k] <= uint32_t(cr.S)) ns += v[k];
            uint32_t ntot;
            uint32_t so = block_exclusive_scan(ns, warps, &ntot);
            if (threadIdx.x == 0) small_base = ntot ? atomicAdd(cr.nsmall, ntot) : 0u;
            __syncthreads();
            uint32_t cs = bs + pre - s;  // pre has advanced past this thread's cells
            if (ntot <= uint32_t(kSmallStage)) {
                // through shared memory, so the list leaves in coalesced runs
                uint32_t w = so;
#pragma unroll
                for (int k = 0; k < per; ++k) {
                    if (v[k] <= uint32_t(cr.S))
                        for (uint32_t q = 0; q < v[k]; ++q) stage[w++] = cs + q;
                    cs += v[k];
                }
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < ntot; i += kSortThreads) cr.small_slots[small_base + i] = stage[i];
            } else {
                uint32_t w = small_base + so;
#pragma unroll
                for (int k = 0; k < per; ++k) {
                    if (v[k] <= uint32_t(cr.S))
                        for (uint32_t q = 0; q < v[k]; ++q) cr.small_slots[w++] = cs + q;
                    cs += v[k];
                }
            }
        }
        __syncthreads();
        for (uint32_t e0 = bs + threadIdx.x; e0 < be; e0 += kSortUnroll * kSortThreads) {
            float4 q[kSortUnroll];
            uint32_t r[kSortUnroll];
#pragma unroll
            for (int u = 0; u < kSortUnroll; ++u) {
                const uint32_t e = e0 + u * kSortThreads;
                if (e < be) q[u] = tmp[e];
            }
#pragma unroll
            for (int u = 0; u < kSortUnroll; ++u)
                if (e0 + u * kSortThreads < be) r[u] = atomicAdd(&hist[local_cell(q[u], g)], 1u);
#pragma unroll
            for (int u = 0; u < kSortUnroll; ++u)
                if (e0 + u * kSortThreads < be) spos[bs + r[u]] = q[u];
        }
        __syncthreads();
    }
}

__global__ void set_u32_kernel(uint32_t *p, uint32_t v) { *p = v; }

void launch_bin_cells(const float *pos, int64_t N, float L, int n, bool wrap, const LinkParams &lp,
                      const FofBuffers &fb, const DevStatus &st, cudaStream_t s) {
    BinGeom g{L, float(double(n) / double(L)), n, bricks_per_axis(n), wrap};
    int64_t n_bricks = int64_t(g.nb) * g.nb * g.nb;
    cudaMemsetAsync(fb.counters, 0, kCounters * sizeof(uint32_t), s);
    const bool few = n_bricks <= kFewBricks;
    const uint32_t *bstart = fb.brick_start;
    int64_t bstride = 1;
    if (few) {
        const int64_t chunk = (N + kFewGrid - 1) / kFewGrid;
        {
            JFOF_TRACE("bin_count", s);
            bin_count_few_kernel<<<kFewGrid, kFewThreads, 0, s>>>(pos, N, g, int(n_bricks), chunk, fb.bin_mat, st);
        }
        {
            JFOF_TRACE("scan", s);
            scan_exclusive(BrickMajor{fb.bin_mat, n_bricks}, n_bricks * kFewGrid, fb.bin_base, fb.scan_tmp, s);
        }
        {
            JFOF_TRACE("bin_scatter", s);
            bin_scatter_few_kernel<<<kFewGrid, kFewThreads, 0, s>>>(pos, N, g, int(n_bricks), chunk, fb.bin_base,
                                                                     fb.tmp, st);
        }
        bstart = fb.bin_base;
        bstride = kFewGrid;
    } else {
        cudaMemsetAsync(fb.brick_count, 0, sizeof(uint32_t) * size_t(n_bricks), s);
        {
            JFOF_TRACE("bin_count", s);
            bin_count_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, g, fb.brick_count, st);
        }
        {
            JFOF_TRACE("scan", s);
            scan_exclusive(LoadU32{fb.brick_count}, n_bricks, fb.brick_start, fb.scan_tmp, s);
        }
        cudaMemcpyAsync(fb.cursor, fb.brick_start, sizeof(uint32_t) * size_t(n_bricks), cudaMemcpyDeviceToDevice,
                        s);
        {
            JFOF_TRACE("bin_scatter", s);
            bin_scatter_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, g, fb.cursor, fb.tmp, st);
        }
    }
    ClassReg cr{lp.S,
                lp.T,
                fb.dense_id,
                fb.dense_cells,
                fb.counters,
                lp.D_cap,
                fb.medium_cells,
                fb.counters + 1,
                fb.counters + 8,
                medium_cap(N),
                lp.S < INT32_MAX ? fb.small_slots : nullptr,
                fb.counters + 6};
    {
        JFOF_TRACE("brick_sort", s);
        brick_sort_kernel<<<grid_for(n_bricks * kSortThreads, kSortThreads, 4), kSortThreads, 0, s>>>(
            fb.tmp, bstart, bstride, n_bricks, g, fb.spos, fb.cell_start, cr);
    }
    set_u32_kernel<<<1, 1, 0, s>>>(fb.cell_start + n_bricks * kBrickCells, uint32_t(N));
}

}  // namespace jfof
