// k_fof.cu -- a1-a6 of the hot path on sm_103a: wrap, cell binning, two-level
// counting sort by cell, the 27-cell neighbour scan fused with lock-free
// union-find, and the raw labels (smallest original index per component).
//
// Layout in HBM (all in the caller's workspace):
//   tmp   float4[N]   particles grouped by brick (16^3 cells), scatter order
//   spos  float4[N]   particles sorted by cell (brick-major), .w = original index
//   cell_start u32[nb^3 * 4096 + 1]   brick-major cell table
//   parent i32[N], rootmin i32[N]     union-find forest over sorted slots (reuse tmp)
#include "jfof_internal.cuh"
#include "k_fof.cuh"

namespace jfof {

// ---------------------------------------------------------------------------
// Pass 1: wrap/check, cell -> brick histogram (L2-resident counters).
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
__global__ void __launch_bounds__(256) bin_scatter_kernel(const float *__restrict__ pos, int64_t N, BinGeom g,
                                                          uint32_t *__restrict__ cursor, float4 *__restrict__ tmp,
                                                          DevStatus st) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        float x, y, z;
        load_particle(pos, i, g, st, x, y, z);
        int ix = cell_coord(x, g.inv_cell, g.n), iy = cell_coord(y, g.inv_cell, g.n), iz = cell_coord(z, g.inv_cell, g.n);
        uint64_t brick = uint64_t(ix >> 4) + uint64_t(g.nb) * (uint64_t(iy >> 4) + uint64_t(g.nb) * uint64_t(iz >> 4));
        uint32_t slot = atomicAdd(&cursor[brick], 1u);
        tmp[slot] = make_float4(x, y, z, __int_as_float(int(i)));
    }
}

// Pass 3: one CTA per brick (persistent loop): shared-memory counting sort of
// the brick's particles by local cell; writes the brick's 4096 cell starts.
constexpr int kSortThreads = 512;

__global__ void __launch_bounds__(kSortThreads) brick_sort_kernel(const float4 *__restrict__ tmp,
                                                                  const uint32_t *__restrict__ brick_start,
                                                                  int64_t n_bricks, BinGeom g,
                                                                  float4 *__restrict__ spos,
                                                                  uint32_t *__restrict__ cell_start) {
    __shared__ uint32_t hist[kBrickCells];
    __shared__ uint32_t warps[kSortThreads / 32];
    constexpr int per = kBrickCells / kSortThreads;  // 8
    for (int64_t brick = blockIdx.x; brick < n_bricks; brick += gridDim.x) {
        uint32_t bs = brick_start[brick], be = brick_start[brick + 1];
        for (int k = threadIdx.x; k < kBrickCells; k += kSortThreads) hist[k] = 0;
        __syncthreads();
        for (uint32_t e = bs + threadIdx.x; e < be; e += kSortThreads) {
            float4 q = tmp[e];
            int ix = cell_coord(q.x, g.inv_cell, g.n), iy = cell_coord(q.y, g.inv_cell, g.n),
                iz = cell_coord(q.z, g.inv_cell, g.n);
            uint32_t lc = uint32_t(ix & 15) + 16u * (uint32_t(iy & 15) + 16u * uint32_t(iz & 15));
            atomicAdd(&hist[lc], 1u);
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
            hist[threadIdx.x * per + k] = pre;
            cell_start[tbase + threadIdx.x * per + k] = bs + pre;
            pre += v[k];
        }
        __syncthreads();
        for (uint32_t e = bs + threadIdx.x; e < be; e += kSortThreads) {
            float4 q = tmp[e];
            int ix = cell_coord(q.x, g.inv_cell, g.n), iy = cell_coord(q.y, g.inv_cell, g.n),
                iz = cell_coord(q.z, g.inv_cell, g.n);
            uint32_t lc = uint32_t(ix & 15) + 16u * (uint32_t(iy & 15) + 16u * uint32_t(iz & 15));
            uint32_t r = atomicAdd(&hist[lc], 1u);
            spos[bs + r] = q;
        }
        __syncthreads();
    }
}

__global__ void set_u32_kernel(uint32_t *p, uint32_t v) { *p = v; }

void launch_bin_cells(const float *pos, int64_t N, float L, int n, bool wrap, const FofBuffers &fb,
                      const DevStatus &st, cudaStream_t s) {
    BinGeom g{L, float(double(n) / double(L)), n, bricks_per_axis(n), wrap};
    int64_t n_bricks = int64_t(g.nb) * g.nb * g.nb;
    cudaMemsetAsync(fb.brick_count, 0, sizeof(uint32_t) * size_t(n_bricks), s);
    {
        JFOF_TRACE("bin_count", s);
        bin_count_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, g, fb.brick_count, st);
    }
    { JFOF_TRACE("scan", s); scan_exclusive(LoadU32{fb.brick_count}, n_bricks, fb.brick_start, fb.scan_tmp, s); }
    cudaMemcpyAsync(fb.cursor, fb.brick_start, sizeof(uint32_t) * size_t(n_bricks), cudaMemcpyDeviceToDevice, s);
    {
        JFOF_TRACE("bin_scatter", s);
        bin_scatter_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, g, fb.cursor, fb.tmp, st);
    }
    {
        JFOF_TRACE("brick_sort", s);
        brick_sort_kernel<<<grid_for(n_bricks * kSortThreads, kSortThreads, 4), kSortThreads, 0, s>>>(
            fb.tmp, fb.brick_start, n_bricks, g, fb.spos, fb.cell_start);
    }
    set_u32_kernel<<<1, 1, 0, s>>>(fb.cell_start + n_bricks * kBrickCells, uint32_t(N));
}

// ---------------------------------------------------------------------------
// a4+a5: neighbour scan fused with union-find.  One thread per sorted slot s:
// pairs (s, j) with j > s inside its own cell, and every particle of the 13
// "forward" neighbour cells (offsets whose first non-zero component of
// (dz, dy, dx) is positive), so each unordered adjacent cell pair is visited
// once.  The predicate is symmetric bit for bit (fl(a-b) = -fl(b-a) and the
// minimum-image correction is sign-symmetric), so testing (s, j) once from
// either side gives the same answer.
struct LinkGeom {
    float L, hL, b2, inv_cell;
    int n, nb;
};

__constant__ int8_t c_fwd[13][3] = {{1, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},  {-1, -1, 1},
                                    {0, -1, 1}, {1, -1, 1}, {-1, 0, 1}, {0, 0, 1},  {1, 0, 1},
                                    {-1, 1, 1}, {0, 1, 1},  {1, 1, 1}};

__global__ void iota_kernel(int *__restrict__ p, int64_t N) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = int(i);
}

__device__ __forceinline__ void scan_range(const float4 *__restrict__ spos, float4 p, int s, uint32_t a, uint32_t e,
                                           const LinkGeom &g, int *parent, const DevStatus &st) {
    for (uint32_t j = a; j < e; ++j) {
        float4 q = spos[j];
        if (pair_d2(p, q, g.L, g.hL) <= g.b2) uf_unite(parent, s, int(j), st);
    }
}

__global__ void __launch_bounds__(256) link_kernel(const float4 *__restrict__ spos,
                                                   const uint32_t *__restrict__ cell_start, int64_t N, LinkGeom g,
                                                   int *parent, DevStatus st) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        float4 p = spos[s];
        int cx = cell_coord(p.x, g.inv_cell, g.n), cy = cell_coord(p.y, g.inv_cell, g.n),
            cz = cell_coord(p.z, g.inv_cell, g.n);
        uint64_t own = cell_table_index(cx, cy, cz, g.nb);
        scan_range(spos, p, int(s), uint32_t(s) + 1, cell_start[own + 1], g, parent, st);
        if (g.n < 3) continue;
#pragma unroll 1
        for (int k = 0; k < 13; ++k) {
            int nx = cx + c_fwd[k][0], ny = cy + c_fwd[k][1], nz = cz + c_fwd[k][2];
            nx = nx < 0 ? nx + g.n : (nx >= g.n ? nx - g.n : nx);
            ny = ny < 0 ? ny + g.n : (ny >= g.n ? ny - g.n : ny);
            nz = nz < 0 ? nz + g.n : (nz >= g.n ? nz - g.n : nz);
            uint64_t c = cell_table_index(nx, ny, nz, g.nb);
            scan_range(spos, p, int(s), cell_start[c], cell_start[c + 1], g, parent, st);
        }
    }
}

// a6: raw labels.  Pass 1 freezes every slot onto its root (read-only finds,
// so the only write to parent[s] is the root) and takes the smallest original
// index per root; pass 2 writes label[orig] in original order.
__global__ void __launch_bounds__(256) finalize_roots_kernel(const float4 *__restrict__ spos, int64_t N, int *parent,
                                                             int *__restrict__ rootmin) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        int r = uf_find_ro(parent, int(s));
        parent[s] = r;
        atomicMin(&rootmin[r], __float_as_int(spos[s].w));
    }
}

__global__ void __launch_bounds__(256) finalize_labels_kernel(const float4 *__restrict__ spos, int64_t N,
                                                              const int *__restrict__ parent,
                                                              const int *__restrict__ rootmin,
                                                              int32_t *__restrict__ label) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        int orig = __float_as_int(spos[s].w);
        label[orig] = rootmin[parent[s]];
    }
}

void launch_link(const jfof_cells &c, int32_t *label, const DevStatus &st, cudaStream_t s) {
    int64_t N = c.n;
    int *parent = reinterpret_cast<int *>(c.scratch);
    int *rootmin = parent + align_up(size_t(N), 64);
    const float4 *spos = reinterpret_cast<const float4 *>(c.spos);
    LinkGeom g{c.L, 0.5f * c.L, host_mul(c.b, c.b), float(double(c.n_axis) / double(c.L)), c.n_axis,
               bricks_per_axis(c.n_axis)};
    {
        JFOF_TRACE("link_init", s);
        iota_kernel<<<grid_for(N, 256), 256, 0, s>>>(parent, N);
    }
    {
        JFOF_TRACE("link", s);
        link_kernel<<<grid_for(N, 256), 256, 0, s>>>(spos, c.cell_start, N, g, parent, st);
    }
    cudaMemsetAsync(rootmin, 0x7f, sizeof(int) * size_t(N), s);
    {
        JFOF_TRACE("finalize_roots", s);
        finalize_roots_kernel<<<grid_for(N, 256), 256, 0, s>>>(spos, N, parent, rootmin);
    }
    {
        JFOF_TRACE("finalize_labels", s);
        finalize_labels_kernel<<<grid_for(N, 256), 256, 0, s>>>(spos, N, parent, rootmin, label);
    }
}

}  // namespace jfof
