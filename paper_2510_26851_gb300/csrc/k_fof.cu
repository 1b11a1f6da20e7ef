// k_fof.cu -- a1-a6 of the hot path on sm_103a: wrap, cell binning, two-level
// counting sort by cell, the neighbour scan fused with lock-free union-find,
// and the raw labels (smallest original index per component).
//
// Layout in HBM (all in the caller's workspace, see fof_layout):
//   tmp        float4[N]  particles grouped by brick (16^3 cells); later the
//                         staging area of the dense-cell sort, then rootmin
//   spos       float4[N]  particles sorted by cell (brick-major); .w = original
//                         index; inside a dense cell also sorted by sub-cell
//   cell_start u32[nb^3 * 4096 + 1]   brick-major cell table
//   parent     i32[N]     union-find forest over sorted slots (parent <= slot)
//   dense_id   u32[cells] id of each dense cell (written only for them)
//   dense_cells u32[D_cap], sub_start u16[D_cap][kSubMax+1]
//
// Linking in two regimes.  Cells of side s >= 1.01 b guarantee that friends
// are in the same or adjacent cells (Sec. 2.2, Algorithm 2, with the grid
// reading of the design notes).  A cell holding more than T particles is
// "dense": its particles are re-sorted by sub-cells of side s_f = s/k with
// sqrt(3) s_f <= b/1.02, so every pair inside one sub-cell is within b under
// the binary32 predicate (the 2% margin dwarfs the ~1e-6 b rounding of the
// cell assignment and of d2); such pairs are linked without being tested.
// Friends then differ by at most 2 sub-cells per axis.  Two sub-cells are
// joined as soon as one tested pair links, and a sub-cell whose root already
// equals the other side's root is skipped.  Every other pair is tested with
// the exact predicate, so the components equal those of testing all pairs.
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
// the brick's particles by local cell; writes the brick's 4096 cell starts and
// registers every cell with more than S particles in the medium or the dense
// work list.
constexpr int kSortThreads = 512;

struct ClassReg {
    int S, T;                 // small: m <= S; dense: T < m <= kDenseMaxM (T = 0: none)
    uint32_t *dense_id;       // [cell table]
    uint32_t *dense_cells;    // [D_cap]
    uint32_t *ndense;         // counter
    int64_t D_cap;
    uint32_t *medium_cells;   // [M_cap]
    uint32_t *nmedium;        // counter
    int64_t M_cap;
};

__global__ void __launch_bounds__(kSortThreads) brick_sort_kernel(const float4 *__restrict__ tmp,
                                                                  const uint32_t *__restrict__ brick_start,
                                                                  int64_t n_bricks, BinGeom g,
                                                                  float4 *__restrict__ spos,
                                                                  uint32_t *__restrict__ cell_start, ClassReg cr) {
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
                    uint32_t id = atomicAdd(cr.nmedium, 1u);
                    if (int64_t(id) < cr.M_cap) cr.medium_cells[id] = uint32_t(gidx);
                }
            }
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

void launch_bin_cells(const float *pos, int64_t N, float L, int n, bool wrap, const LinkParams &lp,
                      const FofBuffers &fb, const DevStatus &st, cudaStream_t s) {
    BinGeom g{L, float(double(n) / double(L)), n, bricks_per_axis(n), wrap};
    int64_t n_bricks = int64_t(g.nb) * g.nb * g.nb;
    cudaMemsetAsync(fb.brick_count, 0, sizeof(uint32_t) * size_t(n_bricks), s);
    cudaMemsetAsync(fb.counters, 0, 2 * sizeof(uint32_t), s);
    {
        JFOF_TRACE("bin_count", s);
        bin_count_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, g, fb.brick_count, st);
    }
    {
        JFOF_TRACE("scan", s);
        scan_exclusive(LoadU32{fb.brick_count}, n_bricks, fb.brick_start, fb.scan_tmp, s);
    }
    cudaMemcpyAsync(fb.cursor, fb.brick_start, sizeof(uint32_t) * size_t(n_bricks), cudaMemcpyDeviceToDevice, s);
    {
        JFOF_TRACE("bin_scatter", s);
        bin_scatter_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, g, fb.cursor, fb.tmp, st);
    }
    ClassReg cr{lp.S, lp.T, fb.dense_id, fb.dense_cells, fb.counters, lp.D_cap, fb.medium_cells, fb.counters + 1,
                medium_cap(N)};
    {
        JFOF_TRACE("brick_sort", s);
        brick_sort_kernel<<<grid_for(n_bricks * kSortThreads, kSortThreads, 4), kSortThreads, 0, s>>>(
            fb.tmp, fb.brick_start, n_bricks, g, fb.spos, fb.cell_start, cr);
    }
    set_u32_kernel<<<1, 1, 0, s>>>(fb.cell_start + n_bricks * kBrickCells, uint32_t(N));
}

// ---------------------------------------------------------------------------
// Link geometry and helpers.
struct LinkGeom {
    float L, hL, b2, inv_cell, inv_fine, cell_side, gap2;
    int n, nb, k, k3, S, T;
    int64_t D_cap;
};

// 13 "forward" cell offsets (first non-zero of (dz, dy, dx) positive) followed
// by their negatives: each unordered pair of adjacent cells is one forward
// offset away from exactly one of its two cells (n >= 3).
__constant__ int8_t c_nb26[26][3] = {
    {1, 0, 0},   {-1, 1, 0}, {0, 1, 0},   {1, 1, 0},   {-1, -1, 1}, {0, -1, 1},  {1, -1, 1},
    {-1, 0, 1},  {0, 0, 1},  {1, 0, 1},   {-1, 1, 1},  {0, 1, 1},   {1, 1, 1},   {-1, 0, 0},
    {1, -1, 0},  {0, -1, 0}, {-1, -1, 0}, {1, 1, -1},  {0, 1, -1},  {-1, 1, -1}, {1, 0, -1},
    {0, 0, -1},  {-1, 0, -1}, {1, -1, -1}, {0, -1, -1}, {-1, -1, -1}};

// 62 forward sub-cell offsets of the 5x5x5 stencil (first non-zero of
// (dz, dy, dx) positive), the 13 with all components in {-1,0,1} first;
// filled on the host at first use.
constexpr int kSubNear = 13;
__constant__ int8_t c_sub62[62][3];

__device__ __forceinline__ void decode_cell(uint32_t gidx, int nb, int &cx, int &cy, int &cz) {
    uint32_t brick = gidx >> 12, local = gidx & 4095u;
    uint32_t bx = brick % uint32_t(nb), by = (brick / uint32_t(nb)) % uint32_t(nb), bz = brick / (uint32_t(nb) * nb);
    cx = int(bx * 16 + (local & 15u));
    cy = int(by * 16 + ((local >> 4) & 15u));
    cz = int(bz * 16 + (local >> 8));
}

__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Sub-cell coordinate of x inside cell c (fine index clamped to the cell).
__device__ __forceinline__ int sub_coord(float x, float inv_fine, int c, int k) {
    int f = __float2int_rd(__fmul_rn(x, inv_fine)) - c * k;
    f = f < 0 ? 0 : f;
    f = f > k - 1 ? k - 1 : f;
    return f;
}

// Cell classes: 0 empty, 1 small, 2 medium, 3 dense.
__device__ __forceinline__ int cell_class(uint32_t m, uint64_t gidx, const LinkGeom &g, const uint32_t *dense_id) {
    if (m == 0) return 0;
    if (m <= uint32_t(g.S)) return 1;
    if (g.T > 0 && m > uint32_t(g.T) && m <= kDenseMaxM && int64_t(dense_id[gidx]) < g.D_cap) return 3;
    return 2;
}

__device__ __forceinline__ bool linked(float4 p, float4 q, const LinkGeom &g) {
    return pair_d2(p, q, g.L, g.hL) <= g.b2;
}

// Squared distance (conservative, float) from a particle to the face/edge/
// corner a neighbour at offset o shares with its own cell c.
__device__ __forceinline__ float gap_to_neighbour(float4 p, int cx, int cy, int cz, int ox, int oy, int oz,
                                                  float side) {
    float gx = ox > 0 ? float(cx + 1) * side - p.x : (ox < 0 ? p.x - float(cx) * side : 0.f);
    float gy = oy > 0 ? float(cy + 1) * side - p.y : (oy < 0 ? p.y - float(cy) * side : 0.f);
    float gz = oz > 0 ? float(cz + 1) * side - p.z : (oz < 0 ? p.z - float(cz) * side : 0.f);
    gx = fmaxf(gx, 0.f);
    gy = fmaxf(gy, 0.f);
    gz = fmaxf(gz, 0.f);
    return gx * gx + gy * gy + gz * gz;
}

__device__ __forceinline__ float4 shfl4(float4 v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// Next task of a warp from a work counter (dynamic scheduling keeps the
// tasks in flight a contiguous window of the work list).
__device__ __forceinline__ int64_t next_task(uint32_t *ctr, int lane) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1u);
    return int64_t(__shfl_sync(0xffffffffu, t, 0));
}

__global__ void iota_kernel(int *__restrict__ p, int64_t N) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = int(i);
}

// ---------------------------------------------------------------------------
// Small cells: one thread per particle.  Pairs with later particles of its
// cell and with every particle of a small forward neighbour cell that lies
// within reach (the particle's gap to that cell <= 1.02 b).  All loops are
// bounded by S.
__global__ void __launch_bounds__(256) small_kernel(const float4 *__restrict__ spos,
                                                    const uint32_t *__restrict__ cell_start, int64_t N, LinkGeom g,
                                                    int *parent, DevStatus st) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        float4 p = spos[s];
        int cx = cell_coord(p.x, g.inv_cell, g.n), cy = cell_coord(p.y, g.inv_cell, g.n),
            cz = cell_coord(p.z, g.inv_cell, g.n);
        uint64_t own = cell_table_index(cx, cy, cz, g.nb);
        uint32_t a1 = cell_start[own + 1];
        if (a1 - cell_start[own] > uint32_t(g.S)) continue;
        for (uint32_t j = uint32_t(s) + 1; j < a1; ++j)
            if (linked(p, spos[j], g)) uf_unite(parent, int(s), int(j), st);
        if (g.n < 3) continue;
#pragma unroll 1
        for (int o = 0; o < 13; ++o) {
            int ox = c_nb26[o][0], oy = c_nb26[o][1], oz = c_nb26[o][2];
            if (gap_to_neighbour(p, cx, cy, cz, ox, oy, oz, g.cell_side) > g.gap2) continue;
            uint64_t nb = cell_table_index(wrapc(cx + ox, g.n), wrapc(cy + oy, g.n), wrapc(cz + oz, g.n), g.nb);
            uint32_t b0 = cell_start[nb], b1 = cell_start[nb + 1];
            if (b1 - b0 > uint32_t(g.S)) continue;  // medium/dense neighbours handle this pair
            for (uint32_t j = b0; j < b1; ++j)
                if (linked(p, spos[j], g)) uf_unite(parent, int(s), int(j), st);
        }
    }
}

// ---------------------------------------------------------------------------
// Path halving in shared memory (each write stores an ancestor of a non-root,
// so concurrent finds and the CAS hook stay correct, as in uf_find).
__device__ __forceinline__ int lfind(volatile int *lp, int x) {
    while (true) {
        int p = lp[x];
        if (p == x) return x;
        int gp = lp[p];
        if (gp == p) return p;
        lp[x] = gp;
        x = gp;
    }
}

__device__ __forceinline__ void lunite(int *lp, int a, int b) {
    for (int it = 0; it < 4 * kSubMax; ++it) {
        int ra = lfind(lp, a), rb = lfind(lp, b);
        if (ra == rb) return;
        if (ra < rb) {
            int t = ra;
            ra = rb;
            rb = t;
        }
        if (atomicCAS(&lp[ra], ra, rb) == ra) return;
    }
}

// ---------------------------------------------------------------------------
// Medium cells, local part: one warp per cell.  The cell's particles are
// staged in shared memory and all their pairs tested in 32-wide tiles
// (lane = one particle, the other broadcast), joined by a shared-memory
// union-find over local indices; then parent[slot] = first slot of the
// slot's local component.  A cell larger than the staging area (possible only
// when it cannot take the dense path) links its own pairs through the global
// forest instead.  Runs before any kernel that unites across cells, since it
// writes parent with plain stores.
constexpr int kMedWarps = 4;
constexpr int kMedCap = 256;

__global__ void __launch_bounds__(32 * kMedWarps) medium_local_kernel(const float4 *__restrict__ spos,
                                                                      const uint32_t *__restrict__ cell_start,
                                                                      const uint32_t *__restrict__ medium_cells,
                                                                      const uint32_t *__restrict__ nmedium,
                                                                      uint32_t *next, int64_t M_cap, LinkGeom g,
                                                                      int *parent, DevStatus st) {
    __shared__ float4 sh_p[kMedWarps][kMedCap];
    __shared__ int sh_l[kMedWarps][kMedCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *sp = sh_p[w];
    int *lp = sh_l[w];
    int64_t M = *nmedium;
    if (M > M_cap) M = M_cap;
    for (int64_t t = next_task(next, lane); t < M; t = next_task(next, lane)) {
        uint32_t ga = medium_cells[t];
        uint32_t a0 = cell_start[ga];
        int mA = int(cell_start[ga + 1] - a0);
        if (mA > kMedCap) {
            for (int i = 0; i < mA - 1; ++i) {
                float4 pi = spos[a0 + i];
                for (int j = i + 1 + lane; j < mA; j += 32)
                    if (linked(pi, spos[a0 + j], g)) uf_unite(parent, int(a0 + i), int(a0 + j), st);
            }
            continue;
        }
        for (int q = lane; q < mA; q += 32) {
            sp[q] = spos[a0 + q];
            lp[q] = q;
        }
        __syncwarp();
        if (mA <= 32) {
            // one particle per lane: 32-bit adjacency masks, same closure
            const bool h0 = lane < mA;
            float4 q0 = h0 ? sp[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned r0 = h0 ? 1u << lane : 0u;
            for (int i = 0; i < mA; ++i)
                if (h0 && linked(sp[i], q0, g)) r0 |= 1u << i;
            for (int round = 0; round < 6; ++round) {
                unsigned n0 = r0;
                for (int i = 0; i < mA; ++i) {
                    unsigned ri = __shfl_sync(0xffffffffu, r0, i);
                    if ((r0 >> i) & 1u) n0 |= ri;
                }
                bool changed = n0 != r0;
                r0 = n0;
                if (!__any_sync(0xffffffffu, changed)) break;
            }
            if (h0) parent[a0 + lane] = int(a0) + __ffs(int(r0)) - 1;
            __syncwarp();
            continue;
        }
        if (mA <= 64) {
            // Warp-synchronous components for up to 64 particles: each lane owns
            // particles lane and lane+32 and builds their 64-bit adjacency masks
            // (every pair tested with the exact predicate), then the reach sets
            // are closed under r_j |= r_i for i in r_j (each round doubles the
            // path length covered) until no mask changes.  The component's
            // smallest local index is the lowest set bit.
            const bool h0 = lane < mA, h1 = lane + 32 < mA;
            float4 q0 = h0 ? sp[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 q1 = h1 ? sp[lane + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned long long r0 = h0 ? 1ull << lane : 0ull, r1 = h1 ? 1ull << (lane + 32) : 0ull;
            for (int i = 0; i < mA; ++i) {
                float4 pi = sp[i];
                if (h0 && linked(pi, q0, g)) r0 |= 1ull << i;
                if (h1 && linked(pi, q1, g)) r1 |= 1ull << i;
            }
            for (int round = 0; round < 8; ++round) {
                unsigned long long n0 = r0, n1 = r1;
                for (int i = 0; i < mA; ++i) {
                    unsigned long long ri = __shfl_sync(0xffffffffu, i < 32 ? r0 : r1, i & 31);
                    if ((r0 >> i) & 1ull) n0 |= ri;
                    if ((r1 >> i) & 1ull) n1 |= ri;
                }
                bool changed = n0 != r0 || n1 != r1;
                r0 = n0;
                r1 = n1;
                if (!__any_sync(0xffffffffu, changed)) break;
            }
            if (h0) parent[a0 + lane] = int(a0) + __ffsll((long long)r0) - 1;
            if (h1) parent[a0 + lane + 32] = int(a0) + __ffsll((long long)r1) - 1;
            __syncwarp();
            continue;
        }
        for (int cb = 0; cb * 32 < mA; ++cb) {
            int j = cb * 32 + lane;
            bool has = j < mA;
            float4 pj = has ? sp[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            int iend = min(mA, cb * 32 + 32) - 1;
            for (int i = 0; i < iend; ++i) {
                float4 pi = sp[i];
                if (has && i < j && linked(pi, pj, g)) lunite(lp, i, j);
            }
        }
        __syncwarp();
        for (int q = lane; q < mA; q += 32) parent[a0 + q] = int(a0) + lfind(lp, q);
        __syncwarp();
    }
}

// Medium cells, cross part: one warp per cell.  For each small neighbour
// (any direction) and each medium forward neighbour, the particles of both
// cells that lie within reach of the shared face/edge/corner are selected by
// ballot and their cross pairs spread over lanes.
__global__ void __launch_bounds__(256) medium_kernel(const float4 *__restrict__ spos,
                                                     const uint32_t *__restrict__ cell_start,
                                                     const uint32_t *__restrict__ medium_cells,
                                                     const uint32_t *__restrict__ nmedium, uint32_t *next,
                                                     const uint32_t *__restrict__ dense_id, int64_t M_cap,
                                                     LinkGeom g, int *parent, DevStatus st) {
    const int lane = threadIdx.x & 31;
    int64_t M = *nmedium;
    if (M > M_cap) M = M_cap;
    for (int64_t t = next_task(next, lane); t < M; t = next_task(next, lane)) {
        uint32_t ga = medium_cells[t];
        int cx, cy, cz;
        decode_cell(ga, g.nb, cx, cy, cz);
        uint32_t a0 = cell_start[ga];
        int mA = int(cell_start[ga + 1] - a0);
        if (g.n < 3) continue;
        uint32_t nb0 = 0, nb1 = 0;
        int ncls = 0;
        if (lane < 26) {
            uint64_t gb = cell_table_index(wrapc(cx + c_nb26[lane][0], g.n), wrapc(cy + c_nb26[lane][1], g.n),
                                           wrapc(cz + c_nb26[lane][2], g.n), g.nb);
            nb0 = cell_start[gb];
            nb1 = cell_start[gb + 1];
            ncls = cell_class(nb1 - nb0, gb, g, dense_id);
        }
        // Cached component representatives of the cell's first 64 particles
        // (lane holds particles lane and lane+32).  Equal representatives
        // mean one component, so such a linked pair needs no union; after a
        // union every cached value naming either side becomes the merged
        // representative.  A stale value only costs an exact union.
        int rep0 = lane < mA ? uf_find(parent, int(a0 + lane)) : -1;
        int rep1 = lane + 32 < mA ? uf_find(parent, int(a0 + lane + 32)) : -1;
        for (int o = 0; o < 26; ++o) {
            int cls = __shfl_sync(0xffffffffu, ncls, o);
            if (cls == 0 || cls == 3 || (cls == 2 && o >= 13)) continue;
            uint32_t b0 = __shfl_sync(0xffffffffu, nb0, o), b1 = __shfl_sync(0xffffffffu, nb1, o);
            int ox = c_nb26[o][0], oy = c_nb26[o][1], oz = c_nb26[o][2];
            int bx = wrapc(cx + ox, g.n), by = wrapc(cy + oy, g.n), bz = wrapc(cz + oz, g.n);
            int mB = int(b1 - b0);
            for (int ca = 0; ca < mA; ca += 32) {
                int i = ca + lane;
                float4 pa = make_float4(0.f, 0.f, 0.f, 0.f);
                bool ina = i < mA;
                if (ina) {
                    pa = spos[a0 + i];
                    ina = gap_to_neighbour(pa, cx, cy, cz, ox, oy, oz, g.cell_side) <= g.gap2;
                }
                unsigned ma = __ballot_sync(0xffffffffu, ina);
                if (!ma) continue;
                for (int cb = 0; cb < mB; cb += 32) {
                    int j = cb + lane;
                    float4 qb = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool inb = j < mB;
                    if (inb) {
                        qb = spos[b0 + j];
                        inb = gap_to_neighbour(qb, bx, by, bz, -ox, -oy, -oz, g.cell_side) <= g.gap2;
                    }
                    if (!__ballot_sync(0xffffffffu, inb)) continue;
                    int repb = inb ? uf_find(parent, int(b0 + j)) : -2;
                    unsigned bits = ma;
                    while (bits) {
                        int src = __ffs(bits) - 1;
                        bits &= bits - 1;
                        float4 x = shfl4(pa, src);
                        int ra = ca == 0 ? __shfl_sync(0xffffffffu, rep0, src)
                                         : (ca == 32 ? __shfl_sync(0xffffffffu, rep1, src) : -3);
                        bool join = inb && ra != repb && linked(x, qb, g);
                        int merged = join ? uf_unite_rep(parent, int(a0 + ca + src), int(b0 + j), st) : 0;
                        unsigned um = __ballot_sync(0xffffffffu, join);
                        while (um) {
                            int L = __ffs(um) - 1;
                            um &= um - 1;
                            int s1 = __shfl_sync(0xffffffffu, ra, L), s2 = __shfl_sync(0xffffffffu, repb, L);
                            int nr = __shfl_sync(0xffffffffu, merged, L);
                            if (rep0 == s1 || rep0 == s2) rep0 = nr;
                            if (rep1 == s1 || rep1 == s2) rep1 = nr;
                            if (repb == s1 || repb == s2) repb = nr;
                        }
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Dense cells, part 1: one warp per dense cell.  Counting sort of the cell's
// particles by sub-cell (staged through tmp), the sub-cell table, then a
// shared-memory union-find over the cell's sub-cells (a sub-cell is one node:
// its members are friends), processing the 13 adjacent forward offsets for
// every non-empty sub-cell first and the other 49 after, with the
// (sub-cell, offset) work spread over lanes; finally
// parent[slot] = first slot of the slot's local component.
constexpr int kDenseWarps = 4;

__device__ __forceinline__ int sub_key(float4 q, const LinkGeom &g, int cx, int cy, int cz) {
    return sub_coord(q.x, g.inv_fine, cx, g.k) +
           g.k * (sub_coord(q.y, g.inv_fine, cy, g.k) + g.k * sub_coord(q.z, g.inv_fine, cz, g.k));
}

// One round of the dense-cell local union-find: every (non-empty sub-cell,
// forward offset O0..O0+R-1) task, spread over the lanes; a task is skipped
// when the two sub-cells are already in one component, else the pair of
// sub-cells is tested until its first link.
template <int O0, int R>
__device__ __forceinline__ void dense_round(const uint32_t *ne, int nF, int k, const uint16_t *ss, int *lp,
                                            const float4 *__restrict__ cp, const LinkGeom &g, int lane,
                                            const int *offs) {
    const int total = nF * R;
    for (int p = lane; p < total; p += 32) {
        uint32_t e = ne[p / R];  // key | x << 10 | y << 14 | z << 18
        int F = int(e & 1023u);
        int o = offs[O0 + p % R];  // (dx+2) | (dy+2) << 3 | (dz+2) << 6
        int gx = int((e >> 10) & 15u) + (o & 7) - 2, gy = int((e >> 14) & 15u) + ((o >> 3) & 7) - 2,
            gz = int((e >> 18) & 15u) + ((o >> 6) & 7) - 2;
        if (unsigned(gx) >= unsigned(k) || unsigned(gy) >= unsigned(k) || unsigned(gz) >= unsigned(k)) continue;
        int G = gx + k * (gy + k * gz);
        int g0 = ss[G], g1 = ss[G + 1];
        if (g0 == g1) continue;
        if (lfind(lp, F) == lfind(lp, G)) continue;
        int f0 = ss[F], f1 = ss[F + 1];
        bool done = false;
        for (int a = f0; a < f1 && !done; ++a) {
            float4 pa = cp[a];
            for (int c = g0; c < g1; ++c) {
                if (linked(pa, cp[c], g)) {
                    lunite(lp, F, G);
                    done = true;
                    break;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(32 * kDenseWarps) dense_cells_kernel(float4 *__restrict__ spos,
                                                                       float4 *__restrict__ stage,
                                                                       const uint32_t *__restrict__ cell_start,
                                                                       const uint32_t *__restrict__ dense_cells,
                                                                       const uint32_t *__restrict__ ndense,
                                                                       uint32_t *next, uint16_t *__restrict__ sub_start,
                                                                       int *__restrict__ parent, LinkGeom g) {
    __shared__ int sh_cnt[kDenseWarps][kSubMax + 1];
    __shared__ uint16_t sh_ss[kDenseWarps][kSubMax + 2];
    __shared__ uint32_t sh_ne[kDenseWarps][kSubMax + 1];
    __shared__ int sh_off[62];
    __shared__ int sh_off2[2 * (62 - kSubNear)];
    __shared__ int sh_sz[kDenseWarps][kSubMax + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *cnt = sh_cnt[w];
    uint16_t *ss = sh_ss[w];
    uint32_t *ne = sh_ne[w];
    int *sz = sh_sz[w];
    for (int o = threadIdx.x; o < 62; o += blockDim.x)
        sh_off[o] = (c_sub62[o][0] + 2) | ((c_sub62[o][1] + 2) << 3) | ((c_sub62[o][2] + 2) << 6);
    for (int o = threadIdx.x; o < 62 - kSubNear; o += blockDim.x) {
        int dx = c_sub62[kSubNear + o][0], dy = c_sub62[kSubNear + o][1], dz = c_sub62[kSubNear + o][2];
        sh_off2[2 * o] = (dx + 2) | ((dy + 2) << 3) | ((dz + 2) << 6);
        sh_off2[2 * o + 1] = (2 - dx) | ((2 - dy) << 3) | ((2 - dz) << 6);
    }
    __syncthreads();
    int64_t D = *ndense;
    if (D > g.D_cap) D = g.D_cap;
    const int k = g.k, k3 = g.k3;
    for (int64_t d = next_task(next, lane); d < D; d = next_task(next, lane)) {
        uint32_t gidx = dense_cells[d];
        uint32_t start = cell_start[gidx];
        int m = int(cell_start[gidx + 1] - start);
        int cx, cy, cz;
        decode_cell(gidx, g.nb, cx, cy, cz);
        for (int key = lane; key < k3; key += 32) cnt[key] = 0;
        __syncwarp();
        for (int t = lane; t < m; t += 32) {
            float4 q = spos[start + t];
            stage[start + t] = q;
            atomicAdd(&cnt[sub_key(q, g, cx, cy, cz)], 1);
        }
        __syncwarp();
        // exclusive scan of the k3 counts (lane owns a contiguous chunk) and
        // the compact list of non-empty sub-cells
        const int chunk = (k3 + 31) / 32;
        int lo = lane * chunk, hi = min(lo + chunk, k3);
        int sum = 0, nz = 0;
        for (int key = lo; key < hi; ++key) {
            sum += cnt[key];
            nz += cnt[key] > 0;
        }
        int xs = sum, xn = nz;
        for (int o = 1; o < 32; o <<= 1) {
            int ys = __shfl_up_sync(0xffffffffu, xs, o), yn = __shfl_up_sync(0xffffffffu, xn, o);
            if (lane >= o) {
                xs += ys;
                xn += yn;
            }
        }
        int pre = xs - sum, pn = xn - nz;
        int nF = __shfl_sync(0xffffffffu, xn, 31);
        uint16_t *tab = sub_start + d * (kSubMax + 1);
        for (int key = lo; key < hi; ++key) {
            int c = cnt[key];
            ss[key] = uint16_t(pre);
            tab[key] = uint16_t(pre);
            cnt[key] = pre;
            if (c > 0) {
                int kz = key / (k * k), ky = (key / k) % k, kx = key % k;
                ne[pn++] = uint32_t(key) | uint32_t(kx) << 10 | uint32_t(ky) << 14 | uint32_t(kz) << 18;
            }
            pre += c;
        }
        if (lane == 0) {
            ss[k3] = uint16_t(m);
            tab[k3] = uint16_t(m);
        }
        __syncwarp();
        for (int t = lane; t < m; t += 32) {
            float4 q = stage[start + t];
            int r = atomicAdd(&cnt[sub_key(q, g, cx, cy, cz)], 1);
            spos[start + r] = q;
        }
        __syncwarp();
        for (int key = lane; key < k3; key += 32) cnt[key] = key;
        __syncwarp();
        dense_round<0, kSubNear>(ne, nF, k, ss, cnt, spos + start, g, lane, sh_off);
        __syncwarp();
        // full compression: every sub-cell points at its root, so the finds of
        // the second round are one load deep
        for (int i = lane; i < nF; i += 32) cnt[ne[i] & 1023u] = lfind(cnt, int(ne[i] & 1023u));
        __syncwarp();
        // The second round (offsets with a component of +-2) can only join
        // sub-cells still in different components.  Every such pair has an end
        // outside the largest component, so the round runs only from the
        // sub-cells outside it, over the far offsets in both directions.
        for (int key = lane; key < k3; key += 32) sz[key] = 0;
        __syncwarp();
        for (int i = lane; i < nF; i += 32) atomicAdd(&sz[cnt[ne[i] & 1023u]], 1);
        __syncwarp();
        int best_c = -1, best_r = -1;
        for (int i = lane; i < nF; i += 32) {
            int F = int(ne[i] & 1023u);
            if (cnt[F] == F && (sz[F] > best_c || (sz[F] == best_c && F < best_r))) {
                best_c = sz[F];
                best_r = F;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            int oc = __shfl_xor_sync(0xffffffffu, best_c, o), orr = __shfl_xor_sync(0xffffffffu, best_r, o);
            if (oc > best_c || (oc == best_c && orr < best_r)) {
                best_c = oc;
                best_r = orr;
            }
        }
        __syncwarp();
        uint32_t *minority = reinterpret_cast<uint32_t *>(sz);
        int nmin = 0;
        for (int base = 0; base < nF; base += 32) {
            int i = base + lane;
            bool out = i < nF && cnt[ne[i] & 1023u] != best_r;
            uint32_t e = i < nF ? ne[i] : 0u;
            unsigned mask = __ballot_sync(0xffffffffu, out);
            __syncwarp();
            if (out) minority[nmin + __popc(mask & ((1u << lane) - 1u))] = e;
            nmin += __popc(mask);
        }
        __syncwarp();
        if (nmin > 0) dense_round<0, 2 * (62 - kSubNear)>(minority, nmin, k, ss, cnt, spos + start, g, lane, sh_off2);
        __syncwarp();
        for (int t = lane; t < m; t += 32) {
            float4 q = spos[start + t];
            parent[start + t] = int(start) + ss[lfind(cnt, sub_key(q, g, cx, cy, cz))];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Dense cells, part 2: one warp per dense cell, its pairs with neighbours.
// Small and medium neighbours (any direction): each neighbour particle within
// reach of the shared face is probed against the cell's sub-cells within 2
// sub-cells of it (lanes over sub-cells): skipped when already in one
// component, else tested until the first link.  Dense forward neighbours:
// every boundary sub-cell of this cell (lanes) against the neighbour's
// sub-cells within reach, the same way.
__global__ void __launch_bounds__(256) dense_nbr_kernel(const float4 *__restrict__ spos,
                                                        const uint32_t *__restrict__ cell_start,
                                                        const uint32_t *__restrict__ dense_cells,
                                                        const uint32_t *__restrict__ ndense, uint32_t *next,
                                                        const uint32_t *__restrict__ dense_id,
                                                        const uint16_t *__restrict__ sub_start, LinkGeom g,
                                                        int *parent, DevStatus st) {
    const int lane = threadIdx.x & 31;
    int64_t D = *ndense;
    if (D > g.D_cap) D = g.D_cap;
    const int k = g.k;
    for (int64_t d = next_task(next, lane); d < D; d = next_task(next, lane)) {
        if (g.n < 3) break;
        uint32_t ga = dense_cells[d];
        int cx, cy, cz;
        decode_cell(ga, g.nb, cx, cy, cz);
        uint32_t a0 = cell_start[ga];
        const uint16_t *ta = sub_start + d * (kSubMax + 1);
        uint32_t nb0 = 0, nb1 = 0, nid = 0;
        int ncls = 0;
        if (lane < 26) {
            uint64_t gb = cell_table_index(wrapc(cx + c_nb26[lane][0], g.n), wrapc(cy + c_nb26[lane][1], g.n),
                                           wrapc(cz + c_nb26[lane][2], g.n), g.nb);
            nb0 = cell_start[gb];
            nb1 = cell_start[gb + 1];
            ncls = cell_class(nb1 - nb0, gb, g, dense_id);
            if (ncls == 3) nid = dense_id[gb];
        }
        for (int o = 0; o < 26; ++o) {
            int cls = __shfl_sync(0xffffffffu, ncls, o);
            if (cls == 0 || (cls == 3 && o >= 13)) continue;
            uint32_t b0 = __shfl_sync(0xffffffffu, nb0, o), b1 = __shfl_sync(0xffffffffu, nb1, o);
            int off[3] = {c_nb26[o][0], c_nb26[o][1], c_nb26[o][2]};
            int bx = wrapc(cx + off[0], g.n), by = wrapc(cy + off[1], g.n), bz = wrapc(cz + off[2], g.n);
            if (cls != 3) {
                int mB = int(b1 - b0);
                for (int cb = 0; cb < mB; cb += 32) {
                    int j = cb + lane;
                    float4 qb = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool inb = j < mB;
                    if (inb) {
                        qb = spos[b0 + j];
                        inb = gap_to_neighbour(qb, bx, by, bz, -off[0], -off[1], -off[2], g.cell_side) <= g.gap2;
                    }
                    unsigned bits = __ballot_sync(0xffffffffu, inb);
                    while (bits) {
                        int src = __ffs(bits) - 1;
                        bits &= bits - 1;
                        float4 q = shfl4(qb, src);
                        int lq[3] = {sub_coord(q.x, g.inv_fine, bx, k), sub_coord(q.y, g.inv_fine, by, k),
                                     sub_coord(q.z, g.inv_fine, bz, k)};
                        int lo[3], n3[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            int c = lq[a] + off[a] * k;  // q's sub-cell in this cell's frame
                            lo[a] = max(c - 2, 0);
                            n3[a] = min(c + 2, k - 1) - lo[a] + 1;
                        }
                        if (n3[0] <= 0 || n3[1] <= 0 || n3[2] <= 0) continue;
                        int nbox = n3[0] * n3[1] * n3[2];
                        int qs = int(b0 + cb + src);
                        for (int t = lane; t < nbox; t += 32) {
                            int G = (lo[0] + t % n3[0]) + k * ((lo[1] + (t / n3[0]) % n3[1]) + k * (lo[2] + t / (n3[0] * n3[1])));
                            uint32_t c0 = ta[G], c1 = ta[G + 1];
                            if (c0 == c1) continue;
                            if (uf_find(parent, qs) == uf_find(parent, int(a0 + c0))) continue;
                            for (uint32_t c = c0; c < c1; ++c)
                                if (linked(q, spos[a0 + c], g)) {
                                    uf_unite(parent, qs, int(a0 + c), st);
                                    break;
                                }
                        }
                    }
                }
                continue;
            }
            const uint16_t *tb = sub_start + int64_t(__shfl_sync(0xffffffffu, nid, o)) * (kSubMax + 1);
            int flo[3], fn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                flo[a] = off[a] > 0 ? k - 2 : 0;
                fn[a] = off[a] != 0 ? 2 : k;
            }
            int nFb = fn[0] * fn[1] * fn[2];
            for (int f = lane; f < nFb; f += 32) {
                int fc[3] = {flo[0] + f % fn[0], flo[1] + (f / fn[0]) % fn[1], flo[2] + f / (fn[0] * fn[1])};
                int F = fc[0] + k * (fc[1] + k * fc[2]);
                uint32_t f0 = ta[F], f1 = ta[F + 1];
                if (f0 == f1) continue;
                int lo[3], hi[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int c = fc[a] - off[a] * k;
                    lo[a] = max(c - 2, 0);
                    hi[a] = min(c + 2, k - 1);
                }
                for (int zz = lo[2]; zz <= hi[2]; ++zz)
                    for (int yy = lo[1]; yy <= hi[1]; ++yy)
                        for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                            int G = xx + k * (yy + k * zz);
                            uint32_t c0 = tb[G], c1 = tb[G + 1];
                            if (c0 == c1) continue;
                            if (uf_find(parent, int(a0 + f0)) == uf_find(parent, int(b0 + c0))) continue;
                            bool done = false;
                            for (uint32_t a = f0; a < f1 && !done; ++a) {
                                float4 p = spos[a0 + a];
                                for (uint32_t c = c0; c < c1; ++c)
                                    if (linked(p, spos[b0 + c], g)) {
                                        uf_unite(parent, int(a0 + a), int(b0 + c), st);
                                        done = true;
                                        break;
                                    }
                            }
                        }
            }
        }
    }
}

// ---------------------------------------------------------------------------
static bool g_sub62_ready[64] = {};

// Fills the constant sub-cell offset table of the current device (a
// synchronous copy: call outside stream capture).
void ensure_link_tables() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || g_sub62_ready[dev]) return;
    int8_t t[62][3];
    int c = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int dz = -2; dz <= 2; ++dz)
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    bool fwd = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                    bool near = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
                    if (!fwd || near != (pass == 0)) continue;
                    t[c][0] = int8_t(dx);
                    t[c][1] = int8_t(dy);
                    t[c][2] = int8_t(dz);
                    ++c;
                }
    cudaMemcpyToSymbol(c_sub62, t, sizeof(t));
    g_sub62_ready[dev] = true;
}

LinkParams make_link_params(int64_t N, float L, float b, int n, int S, int T) {
    LinkParams lp{};
    double s = double(L) / n;
    int k = int(std::ceil(s * std::sqrt(3.0) * 1.02 / double(b)));
    if (k < 1) k = 1;
    double sf = s / k;
    double eps = 4.0 * double(L) * std::ldexp(1.0, -24);
    bool ok = T > 0 && n >= 5 && k <= kSubSide && std::sqrt(3.0) * (sf + 2 * eps) <= double(b) * (1 - 1e-4) &&
              (double(b) + 2 * eps) / sf < 2.0;
    lp.S = S < 0 ? 0 : S;
    lp.T = ok ? (T > lp.S ? T : lp.S + 1) : 0;
    lp.k = k;
    lp.inv_fine = float(double(n) * k / double(L));
    lp.D_cap = ok ? dense_cap(N) : 0;
    return lp;
}

void launch_link_core(const jfof_cells &c, const FofBuffers &fb, const LinkParams &lp, const DevStatus &st,
                      cudaStream_t s) {
    int64_t N = c.n;
    ensure_link_tables();
    float b2 = host_mul(c.b, c.b);
    double gap = 1.02 * double(c.b);
    LinkGeom g{c.L, 0.5f * c.L, b2, float(double(c.n_axis) / double(c.L)), lp.inv_fine,
               float(double(c.L) / c.n_axis), float(gap * gap), c.n_axis, bricks_per_axis(c.n_axis), lp.k,
               lp.k * lp.k * lp.k, lp.S, lp.T, lp.D_cap};
    const float4 *spos = reinterpret_cast<const float4 *>(c.spos);
    {
        JFOF_TRACE("link_init", s);
        iota_kernel<<<grid_for(N, 256), 256, 0, s>>>(fb.parent, N);
    }
    cudaMemsetAsync(fb.counters + 2, 0, 4 * sizeof(uint32_t), s);  // work counters
    // local passes first: they write parent with plain stores, each for its own cell
    if (lp.T > 0) {
        JFOF_TRACE("dense_cells", s);
        dense_cells_kernel<<<grid_for(lp.D_cap * 32, 32 * kDenseWarps, 8), 32 * kDenseWarps, 0, s>>>(
            fb.spos, fb.tmp, c.cell_start, fb.dense_cells, fb.counters, fb.counters + 2, fb.sub_start, fb.parent, g);
    }
    {
        JFOF_TRACE("link_medium_local", s);
        medium_local_kernel<<<grid_for(medium_cap(N) * 32, 32 * kMedWarps, 8), 32 * kMedWarps, 0, s>>>(
            spos, c.cell_start, fb.medium_cells, fb.counters + 1, fb.counters + 3, medium_cap(N), g, fb.parent, st);
    }
    // then everything that unites across cells (atomic hooks only)
    if (lp.S > 0) {
        JFOF_TRACE("link_small", s);
        small_kernel<<<grid_full(N, 256), 256, 0, s>>>(spos, c.cell_start, N, g, fb.parent, st);
    }
    {
        JFOF_TRACE("link_medium", s);
        medium_kernel<<<grid_for(medium_cap(N) * 32, 256, 8), 256, 0, s>>>(
            spos, c.cell_start, fb.medium_cells, fb.counters + 1, fb.counters + 4, fb.dense_id, medium_cap(N), g,
            fb.parent, st);
    }
    if (lp.T > 0) {
        JFOF_TRACE("link_dense_nbr", s);
        dense_nbr_kernel<<<grid_for(lp.D_cap * 32, 256, 8), 256, 0, s>>>(
            spos, c.cell_start, fb.dense_cells, fb.counters, fb.counters + 5, fb.dense_id, fb.sub_start, g, fb.parent,
            st);
    }
}

void launch_link(const jfof_cells &c, const FofBuffers &fb, const LinkParams &lp, int32_t *label,
                 const DevStatus &st, cudaStream_t s) {
    launch_link_core(c, fb, lp, st, s);
    launch_tail_labels(fb, c.n, label, s);
}

}  // namespace jfof
