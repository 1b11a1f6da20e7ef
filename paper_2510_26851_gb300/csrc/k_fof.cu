// k_fof.cu -- a4-a6 of the hot path on sm_103a: the neighbour scan fused
// with lock-free union-find, and the raw labels (smallest original index per
// component).  Wrapping, binning and the sort by cell are in k_bin.cu.
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
//   sub_rows   u16[D_cap][k_max^2]  occupancy rows of each dense cell's sub-cells
//
// Linking in two regimes.  Cells of side s >= 1.01 b guarantee that friends
// are in the same or adjacent cells (Sec. 2.2, Algorithm 2: the linked-cell
// grid with cells no narrower than the linking length).  A cell holding more than T particles is
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

// The same test without the minimum-image correction.  It is bit-identical
// to linked() whenever |x_j - x_i| <= L/2 on every axis, since the
// correction then leaves each difference unchanged: for two particles of one
// cell when n >= 3 (cells are at most L/3 wide) and for a cell and a
// neighbour that does not wrap around the box when n >= 5 (they lie within
// two cells, at most 2L/5).
__device__ __forceinline__ bool linked_near(float4 p, float4 q, const LinkGeom &g) {
    const float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) <= g.b2;
}

__device__ __forceinline__ bool linked_if(bool near, float4 p, float4 q, const LinkGeom &g) {
    return near ? linked_near(p, q, g) : linked(p, q, g);
}

// Every neighbour of cell (cx, cy, cz) lies within the box without wrapping.
__device__ __forceinline__ bool interior_cell(int cx, int cy, int cz, const LinkGeom &g) {
    return g.n >= 5 && cx >= 1 && cy >= 1 && cz >= 1 && cx <= g.n - 2 && cy <= g.n - 2 && cz <= g.n - 2;
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
// Small cells: a warp takes 32 consecutive entries of the list of particles of
// small cells (written by the brick sort, in cell order).  Each lane finds its
// particle's candidates: the later particles of its own cell and every
// particle of a small forward neighbour cell that lies within reach (the
// particle's gap to that cell <= 1.02 b).  The 13 forward offsets are
// compile-time constants (packed 2 bits per offset and axis, value + 1), so
// the reach test of each is two adds and a compare on the particle's squared
// gaps to its cell's six faces.  The (particle, candidate) pairs of the whole
// warp are then laid out as flat tasks (the warp task runner) and tested by
// all lanes in turn, so no lane idles while another walks a longer list.  All
// lists are bounded by S.
constexpr uint32_t kFwdX = 0x2492492u, kFwdY = 0x2a540a9u, kFwdZ = 0x2aaaa55u;
constexpr int kSmallWarps = 8;
constexpr int kSmallTaskCap = 256;

__device__ __forceinline__ int fwd_comp(uint32_t packed, int o) { return int((packed >> (2 * o)) & 3u) - 1; }

template <class Emit, class Work>
__device__ __forceinline__ void warp_tasks(int c, uint32_t *buf, int cap, int lane, Emit emit, Work work);

__global__ void __launch_bounds__(32 * kSmallWarps) small_kernel(const float4 *__restrict__ spos,
                                                                 const uint32_t *__restrict__ cell_start,
                                                                 const uint32_t *__restrict__ small_slots,
                                                                 const uint32_t *__restrict__ nsmall, uint32_t *next,
                                                                 LinkGeom g, int *parent, DevStatus st) {
    __shared__ float4 sh_p[kSmallWarps][32];
    __shared__ int sh_s[kSmallWarps][32];
    __shared__ uint32_t sh_near[kSmallWarps][32];
    __shared__ uint32_t sh_start[kSmallWarps][32][14];  // [0]: own cell after the particle; [1 + o]: neighbour o
    __shared__ uint8_t sh_cnt[kSmallWarps][32][14];
    __shared__ uint32_t sh_task[kSmallWarps][kSmallTaskCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t(*start)[14] = sh_start[w];
    uint8_t(*cnt)[14] = sh_cnt[w];
    const int64_t ns = *nsmall;
    for (int64_t c = next_task(next, lane); c * 32 < ns; c = next_task(next, lane)) {
        const int64_t t = c * 32 + lane;
        int total = 0;
        uint32_t used = 0u;  // lists with at least one candidate
        if (t < ns) {
            const int64_t s = small_slots[t];
            const float4 p = spos[s];
            const int cx = cell_coord(p.x, g.inv_cell, g.n), cy = cell_coord(p.y, g.inv_cell, g.n),
                      cz = cell_coord(p.z, g.inv_cell, g.n);
            const uint64_t own = cell_table_index(cx, cy, cz, g.nb);
            const uint32_t a1 = cell_start[own + 1];
            if (a1 - cell_start[own] <= uint32_t(g.S)) {
                sh_p[w][lane] = p;
                sh_s[w][lane] = int(s);
                uint32_t nearm = g.n >= 3 ? 1u : 0u;  // pairs of one cell
                start[lane][0] = uint32_t(s) + 1;
                cnt[lane][0] = uint8_t(a1 - uint32_t(s) - 1);
                total = int(a1 - uint32_t(s) - 1);
                if (total > 0) used |= 1u;
                if (g.n >= 3) {
                    // squared gaps to the low and high faces of the cell (as in gap_to_neighbour)
                    float lx = fmaxf(p.x - float(cx) * g.cell_side, 0.f), hx = fmaxf(float(cx + 1) * g.cell_side - p.x, 0.f);
                    float ly = fmaxf(p.y - float(cy) * g.cell_side, 0.f), hy = fmaxf(float(cy + 1) * g.cell_side - p.y, 0.f);
                    float lz = fmaxf(p.z - float(cz) * g.cell_side, 0.f), hz = fmaxf(float(cz + 1) * g.cell_side - p.z, 0.f);
                    lx *= lx;
                    hx *= hx;
                    ly *= ly;
                    hy *= hy;
                    lz *= lz;
                    hz *= hz;
                    uint32_t cand = 0u;
#pragma unroll
                    for (int o = 0; o < 13; ++o) {
                        const int ox = fwd_comp(kFwdX, o), oy = fwd_comp(kFwdY, o), oz = fwd_comp(kFwdZ, o);
                        float d = (ox > 0 ? hx : (ox < 0 ? lx : 0.f)) + (oy > 0 ? hy : (oy < 0 ? ly : 0.f)) +
                                  (oz > 0 ? hz : (oz < 0 ? lz : 0.f));
                        if (d <= g.gap2) cand |= 1u << o;
                    }
                    while (cand) {
                        const int o = __ffs(int(cand)) - 1;
                        cand &= cand - 1u;
                        const int ox = fwd_comp(kFwdX, o), oy = fwd_comp(kFwdY, o), oz = fwd_comp(kFwdZ, o);
                        const uint64_t nb =
                            cell_table_index(wrapc(cx + ox, g.n), wrapc(cy + oy, g.n), wrapc(cz + oz, g.n), g.nb);
                        const uint32_t b0 = cell_start[nb], b1 = cell_start[nb + 1];
                        if (b1 == b0 || b1 - b0 > uint32_t(g.S)) continue;  // medium/dense neighbours handle it
                        start[lane][1 + o] = b0;
                        cnt[lane][1 + o] = uint8_t(b1 - b0);
                        total += int(b1 - b0);
                        used |= 2u << o;
                        if (g.n >= 5 && unsigned(cx + ox) < unsigned(g.n) && unsigned(cy + oy) < unsigned(g.n) &&
                            unsigned(cz + oz) < unsigned(g.n))
                            nearm |= 2u << o;
                    }
                }
                sh_near[w][lane] = nearm;
            }
        }
        __syncwarp();
        // task = lane | list << 5 | index in the list << 9
        warp_tasks(
            total, sh_task[w], kSmallTaskCap, lane,
            [&](auto put) {
                for (uint32_t u = used; u; u &= u - 1u) {
                    const int l = __ffs(int(u)) - 1;
                    for (int k = 0; k < cnt[lane][l]; ++k) put(uint32_t(lane) | uint32_t(l) << 5 | uint32_t(k) << 9);
                }
            },
            [&](uint32_t tk) {
                const int ql = int(tk & 31u), l = int((tk >> 5) & 15u), k = int(tk >> 9);
                const uint32_t j = start[ql][l] + uint32_t(k);
                if (linked_if((sh_near[w][ql] >> l) & 1u, sh_p[w][ql], spos[j], g))
                    uf_unite(parent, sh_s[w][ql], int(j), st);
            });
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
// Components of a cell of at most 32 R particles (staged in sp): lane owns
// particles lane + 32 h (h < R) and one adjacency row of R 32-bit words each
// (word indices are compile-time constants, so the rows stay in registers).
// Every unordered pair is tested once, with the exact predicate, and recorded
// in one of its two rows: inside a word block, lane L tests the particles
// L+1 .. L+16 of the block (indices mod 32); between blocks, the particle of
// the higher block tests all of the lower block.  Components by breadth-first
// search from the lowest unvisited particle: the neighbours of a frontier are
// the bits of the frontier's rows (one warp OR-reduction per word) and the
// particles whose own rows meet the frontier (one ballot per word); the seed
// is the component's smallest local index.  Writes parent[a0 + i] = a0 + seed
// of i's component.
template <int R, bool NEAR>
__device__ __forceinline__ void local_bitmask(const float4 *sp, int mA, uint32_t a0, int lane, const LinkGeom &g,
                                              int *parent) {
    float4 q[R];
    bool hv[R];
    uint32_t r[R][R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        hv[h] = lane + 32 * h < mA;
        q[h] = hv[h] ? sp[lane + 32 * h] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int wd = 0; wd < R; ++wd) r[h][wd] = 0u;
    }
#pragma unroll
    for (int h = 0; h < R; ++h) {
        // inside block h: the 16 particles after this lane's (cyclically)
#pragma unroll 4
        for (int d = 1; d <= 16; ++d) {
            const int jl = (lane + d) & 31, j = 32 * h + jl;
            if (hv[h] && j < mA && linked_if(NEAR, sp[j], q[h], g)) r[h][h] |= 1u << jl;
        }
        // lower blocks: every particle
#pragma unroll
        for (int wi = 0; wi < h; ++wi)
#pragma unroll 4
            for (int i = 32 * wi; i < 32 * wi + 32; ++i)
                if (hv[h] && linked_if(NEAR, sp[i], q[h], g)) r[h][wi] |= 1u << (i & 31);
    }
    uint32_t unv[R];
    int root[R];
#pragma unroll
    for (int wd = 0; wd < R; ++wd) {
        const int c = min(max(mA - 32 * wd, 0), 32);
        unv[wd] = c == 32 ? 0xffffffffu : (1u << c) - 1u;
        root[wd] = 0;
    }
    while (true) {
        int sw = -1;
        uint32_t su = 0u;
#pragma unroll
        for (int wd = R - 1; wd >= 0; --wd)
            if (unv[wd]) {
                sw = wd;
                su = unv[wd];
            }
        if (sw < 0) break;
        const int sb = __ffs(int(su)) - 1, seed = 32 * sw + sb;
        uint32_t comp[R], fr[R];
#pragma unroll
        for (int wd = 0; wd < R; ++wd) comp[wd] = fr[wd] = wd == sw ? 1u << sb : 0u;
        while (true) {
            uint32_t any = 0u;
#pragma unroll
            for (int wd = 0; wd < R; ++wd) any |= fr[wd];
            if (!any) break;
            uint32_t nb[R];
#pragma unroll
            for (int wd = 0; wd < R; ++wd) {
                uint32_t v = 0u;
#pragma unroll
                for (int h = 0; h < R; ++h)
                    if ((fr[h] >> lane) & 1u) v |= r[h][wd];
                nb[wd] = __reduce_or_sync(0xffffffffu, v);
            }
#pragma unroll
            for (int h = 0; h < R; ++h) {
                uint32_t meet = 0u;
#pragma unroll
                for (int wd = 0; wd < R; ++wd) meet |= r[h][wd] & fr[wd];
                nb[h] |= __ballot_sync(0xffffffffu, meet != 0u);
            }
#pragma unroll
            for (int wd = 0; wd < R; ++wd) {
                fr[wd] = nb[wd] & ~comp[wd];
                comp[wd] |= nb[wd];
            }
        }
#pragma unroll
        for (int h = 0; h < R; ++h) {
            if ((comp[h] >> lane) & 1u) root[h] = seed;
            unv[h] &= ~comp[h];
        }
    }
#pragma unroll
    for (int h = 0; h < R; ++h)
        if (hv[h]) parent[a0 + lane + 32 * h] = int(a0) + root[h];
}

// Medium cells, local part: one warp per cell.  The cell's particles are
// staged in shared memory and all their pairs tested (lane = one particle,
// the other broadcast).  Up to kMedBig particles: adjacency bitmasks, every
// pair tested once, and a breadth-first search over them; larger cells: a shared-memory union-find
// over local indices.  Then parent[slot] = first slot of the slot's local
// component.  A cell larger than the staging area (possible only when it
// cannot take the dense path) links its own pairs through the global forest
// instead.  Cells of at most kMedMain particles come from the front of the
// medium-cell array (LARGE false), larger ones from its back (LARGE true), so
// each instance keeps the registers of its own sizes.
// Runs before any kernel that unites across cells, since it writes parent
// with plain stores.
constexpr int kMedWarps = 4;  // default warps per CTA (the autotuner may pick 8)
constexpr int kMedCap = 256;

template <int W, bool NEAR, bool LARGE>
__global__ void __launch_bounds__(32 * W) medium_local_kernel(const float4 *__restrict__ spos,
                                                                      const uint32_t *__restrict__ cell_start,
                                                                      const uint32_t *__restrict__ medium_cells,
                                                                      const uint32_t *__restrict__ nmedium,
                                                                      uint32_t *next, int64_t M_cap, LinkGeom g,
                                                                      int *parent, DevStatus st) {
    __shared__ float4 sh_p[W][kMedCap];
    __shared__ int sh_l[W][kMedCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *sp = sh_p[w];
    int *lp = sh_l[w];
    int64_t M = *nmedium;
    if (M > M_cap) M = M_cap;
    for (int64_t t = next_task(next, lane); t < M; t = next_task(next, lane)) {
        uint32_t ga = medium_cells[LARGE ? M_cap - 1 - t : t];
        uint32_t a0 = cell_start[ga];
        int mA = int(cell_start[ga + 1] - a0);
        if (mA > kMedCap) {
            for (int i = 0; i < mA - 1; ++i) {
                float4 pi = spos[a0 + i];
                for (int j = i + 1 + lane; j < mA; j += 32)
                    if (linked_if(NEAR, pi, spos[a0 + j], g)) uf_unite(parent, int(a0 + i), int(a0 + j), st);
            }
            continue;
        }
        for (int q = lane; q < mA; q += 32) {
            sp[q] = spos[a0 + q];
            lp[q] = q;
        }
        __syncwarp();
        if (!LARGE && mA <= 32) {
            local_bitmask<1, NEAR>(sp, mA, a0, lane, g, parent);
            __syncwarp();
            continue;
        }
        if (!LARGE && mA <= 64) {
            local_bitmask<2, NEAR>(sp, mA, a0, lane, g, parent);
            __syncwarp();
            continue;
        }
        if (!LARGE && mA <= kMedMain) {
            local_bitmask<3, NEAR>(sp, mA, a0, lane, g, parent);
            __syncwarp();
            continue;
        }
        if (LARGE && mA <= 128) {
            local_bitmask<4, NEAR>(sp, mA, a0, lane, g, parent);
            __syncwarp();
            continue;
        }
        if (LARGE && mA <= kMedBig) {
            local_bitmask<5, NEAR>(sp, mA, a0, lane, g, parent);
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
                if (has && i < j && linked_if(NEAR, pi, pj, g)) lunite(lp, i, j);
            }
        }
        __syncwarp();
        for (int q = lane; q < mA; q += 32) parent[a0 + q] = int(a0) + lfind(lp, q);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Warp task runner: every lane brings c tasks (emit(put) hands them to put in
// a fixed order); the warp lays them out in a shared-memory window of cap
// entries at a time and all lanes then take them in turn (work(task)).
template <class Emit, class Work>
__device__ __forceinline__ void warp_tasks(int c, uint32_t *buf, int cap, int lane, Emit emit, Work work) {
    int pre = c;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    pre -= c;
    for (int w0 = 0; w0 < total; w0 += cap) {
        if (c > 0 && pre < w0 + cap && pre + c > w0) {
            int idx = pre;
            emit([&](uint32_t task) {
                if (idx >= w0 && idx < w0 + cap) buf[idx - w0] = task;
                ++idx;
            });
        }
        __syncwarp();
        const int nt = min(cap, total - w0);
        for (int t = lane; t < nt; t += 32) work(buf[t]);
        __syncwarp();
    }
}

// Box of sub-cells, inclusive per axis.
struct SubBox {
    int x0, y0, z0, x1, y1, z1;
};

// Medium cells, cross part: one warp per cell A.  Every particle of a small
// neighbour (any direction) or a medium forward neighbour that lies within
// reach of A is gathered, with the offset of its cell, into a shared-memory
// list (the neighbours' particles are spread over the lanes as one flat
// range); the list is then swept one entry per lane over the particles of A
// that reach the entry's offset (a 26-bit reach mask per particle, and per
// offset the set of particles that reach it).  Cached
// component representatives (one per particle of A, one per entry): a value
// is always a node that was in the entity's component at some time, so equal
// values mean one component and such a linked pair needs no union; a union
// stores the merged representative on both sides (a stale value only costs
// an exact union).  Cells of at most kMedMain particles come from the front of
// the medium-cell array (LARGE false: reach sets of 3 words), larger ones from
// its back (LARGE true: 5 words, up to kMedBig particles); a cell larger than
// that (possible only when it cannot take the dense path) walks its
// neighbours one at a time instead.
constexpr int kMedXWarps = 8;  // default warps per CTA (the autotuner may pick 4)
constexpr int kMedList = 64;

// Offsets o in cand whose neighbour cell p can reach (gap <= 1.02 b).
__device__ __forceinline__ uint32_t reach_mask(float4 p, int cx, int cy, int cz, uint32_t cand, const LinkGeom &g) {
    // squared gaps to the low and high faces of the cell; offset o and its
    // opposite o + 13 add the gaps of the faces they cross (compile-time
    // offsets, as in the small-cell kernel)
    float lx = fmaxf(p.x - float(cx) * g.cell_side, 0.f), hx = fmaxf(float(cx + 1) * g.cell_side - p.x, 0.f);
    float ly = fmaxf(p.y - float(cy) * g.cell_side, 0.f), hy = fmaxf(float(cy + 1) * g.cell_side - p.y, 0.f);
    float lz = fmaxf(p.z - float(cz) * g.cell_side, 0.f), hz = fmaxf(float(cz + 1) * g.cell_side - p.z, 0.f);
    lx *= lx;
    hx *= hx;
    ly *= ly;
    hy *= hy;
    lz *= lz;
    hz *= hz;
    uint32_t m = 0u;
#pragma unroll
    for (int o = 0; o < 13; ++o) {
        const int ox = fwd_comp(kFwdX, o), oy = fwd_comp(kFwdY, o), oz = fwd_comp(kFwdZ, o);
        const float d = (ox > 0 ? hx : (ox < 0 ? lx : 0.f)) + (oy > 0 ? hy : (oy < 0 ? ly : 0.f)) +
                        (oz > 0 ? hz : (oz < 0 ? lz : 0.f));
        const float e = (ox > 0 ? lx : (ox < 0 ? hx : 0.f)) + (oy > 0 ? ly : (oy < 0 ? hy : 0.f)) +
                        (oz > 0 ? lz : (oz < 0 ? hz : 0.f));
        if (d <= g.gap2) m |= 1u << o;
        if (e <= g.gap2) m |= 1u << (o + 13);
    }
    return m & cand;
}

template <int W, bool LARGE>
__global__ void __launch_bounds__(32 * W) medium_kernel(const float4 *__restrict__ spos,
                                                                 const uint32_t *__restrict__ cell_start,
                                                                 const uint32_t *__restrict__ medium_cells,
                                                                 const uint32_t *__restrict__ nmedium,
                                                                 uint32_t *next,
                                                                 const uint32_t *__restrict__ dense_id,
                                                                 int64_t M_cap, LinkGeom g, int *parent,
                                                                 DevStatus st) {
    __shared__ float4 sh_q[W][kMedList];
    __shared__ int sh_slot[W][kMedList];
    __shared__ int sh_rep[W][kMedList];
    __shared__ int sh_pre[W][32];
    constexpr int R = LARGE ? 5 : 3;                    // words of a reach set
    constexpr int LIM = LARGE ? kMedBig : kMedMain;     // cells the list path takes
    __shared__ float4 sh_pa[W][LIM];
    __shared__ int sh_repa[W][LIM];
    __shared__ uint32_t sh_amask[W][26][R];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *lq = sh_q[w];
    int *lslot = sh_slot[w], *lrep = sh_rep[w], *pre = sh_pre[w];
    float4 *spa = sh_pa[w];
    int *repa = sh_repa[w];
    uint32_t(*amask)[R] = sh_amask[w];
    // this lane's neighbour offset (lanes < 26), packed for shuffles
    const int my_off = lane < 26 ? (c_nb26[lane][0] + 1) | (c_nb26[lane][1] + 1) << 2 | (c_nb26[lane][2] + 1) << 4
                                 : 0;
    int64_t M = *nmedium;
    if (M > M_cap) M = M_cap;
    for (int64_t t = next_task(next, lane); t < M; t = next_task(next, lane)) {
        uint32_t ga = medium_cells[LARGE ? M_cap - 1 - t : t];
        int cx, cy, cz;
        decode_cell(ga, g.nb, cx, cy, cz);
        const uint32_t a0 = cell_start[ga];
        const int mA = int(cell_start[ga + 1] - a0);
        if (g.n < 3) continue;
        const bool near = interior_cell(cx, cy, cz, g);
        uint32_t nb0 = 0, nb1 = 0;
        int ncls = 0;
        if (lane < 26) {
            uint64_t gb = cell_table_index(wrapc(cx + c_nb26[lane][0], g.n), wrapc(cy + c_nb26[lane][1], g.n),
                                           wrapc(cz + c_nb26[lane][2], g.n), g.nb);
            nb0 = cell_start[gb];
            nb1 = cell_start[gb + 1];
            ncls = cell_class(nb1 - nb0, gb, g, dense_id);
        }
        int rep0 = lane < mA ? uf_find(parent, int(a0 + lane)) : -1;
        int rep1 = lane + 32 < mA ? uf_find(parent, int(a0 + lane + 32)) : -1;
        if (mA <= LIM) {
            // neighbours to visit: small cells all round, medium forward
            const uint32_t cand = __ballot_sync(0xffffffffu, lane < 26 && (ncls == 1 || (ncls == 2 && lane < 13)));
            // the cell's particles, their representatives, their reach masks, and
            // per offset the set of particles that reach it (R 32-bit words)
            uint32_t mm[R];
            uint32_t any = 0u;
#pragma unroll
            for (int h = 0; h < R; ++h) {
                const bool in = lane + 32 * h < mA;
                const int rp = h == 0 ? rep0 : (h == 1 ? rep1 : (in ? uf_find(parent, int(a0 + lane + 32 * h)) : -1));
                const float4 pa = in ? spos[a0 + lane + 32 * h] : make_float4(0.f, 0.f, 0.f, 0.f);
                mm[h] = in ? reach_mask(pa, cx, cy, cz, cand, g) : 0u;
                any |= mm[h];
                if (in) {
                    spa[lane + 32 * h] = pa;
                    repa[lane + 32 * h] = rp;
                }
            }
            const uint32_t reach = __reduce_or_sync(0xffffffffu, any);
            for (uint32_t rb = reach; rb; rb &= rb - 1u) {
                const int o = __ffs(int(rb)) - 1;
#pragma unroll
                for (int h = 0; h < R; ++h) {
                    const uint32_t wv = __ballot_sync(0xffffffffu, (mm[h] >> o) & 1u);
                    if (lane == 0) amask[o][h] = wv;
                }
            }
            const bool take = (reach >> lane) & 1u;
            const int c = take ? int(nb1 - nb0) : 0;
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            pre[lane] = incl;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            int nl = 0;
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int tt = t0 + lane;
                // owner neighbour: number of inclusive prefixes <= tt
                int o = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (pre[o + step - 1] <= tt) o += step;
                const int src = tt < total ? o : 0;
                const uint32_t ob0 = __shfl_sync(0xffffffffu, nb0, src);
                const int opk = __shfl_sync(0xffffffffu, my_off, src);
                const int ex = __shfl_sync(0xffffffffu, incl - c, src);
                bool inb = tt < total;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                int qs = 0;
                if (inb) {
                    const int ox = (opk & 3) - 1, oy = ((opk >> 2) & 3) - 1, oz = ((opk >> 4) & 3) - 1;
                    qs = int(ob0) + (tt - ex);
                    q = spos[qs];
                    inb = gap_to_neighbour(q, wrapc(cx + ox, g.n), wrapc(cy + oy, g.n), wrapc(cz + oz, g.n), -ox, -oy,
                                           -oz, g.cell_side) <= g.gap2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, inb);
                if (inb) {
                    int pos = nl + __popc(bal & ((1u << lane) - 1u));
                    lq[pos] = make_float4(q.x, q.y, q.z, __int_as_float(src));
                    lslot[pos] = qs;
                }
                nl += __popc(bal);
                __syncwarp();
                if (nl > kMedList - 32 || (t0 + 32 >= total && nl > 0)) {
                    // sweep the list: each entry against the particles of A that
                    // reach its offset
                    for (int e = lane; e < nl; e += 32) lrep[e] = uf_find(parent, lslot[e]);
                    __syncwarp();
                    // One entry per lane, its reaching particles in turn: once
                    // the entry has joined a component, the particles of A
                    // already known to be in it cost one comparison each
                    // (their cached representative equals the entry's, or one
                    // of the last representatives the entry's unions merged
                    // away).  Flat (entry, particle) tasks spread over the lanes
                    // tested many pairs of one entry at once, before any link
                    // of that entry was visible.
                    for (int e = lane; e < nl; e += 32) {
                        const int oe = __float_as_int(lq[e].w);
                        const float4 qe = lq[e];
                        int re = lrep[e], al0 = -1, al1 = -1, al2 = -1;
#pragma unroll
                        for (int wd = 0; wd < R; ++wd)
                            for (uint32_t bits = amask[oe][wd]; bits; bits &= bits - 1u) {
                                const int ta = 32 * wd + __ffs(int(bits)) - 1;
                                const int ra = repa[ta];
                                if (ra == re || ra == al0 || ra == al1 || ra == al2) continue;
                                if (linked_if(near, spa[ta], qe, g)) {
                                    const int m = uf_unite_rep(parent, int(a0) + ta, lslot[e], st);
                                    repa[ta] = m;
                                    al2 = al1;
                                    al1 = ra;
                                    al0 = re;
                                    re = m;
                                }
                            }
                        lrep[e] = re;
                    }
                    __syncwarp();
                    nl = 0;
                }
            }
            continue;
        }
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
                        bool join = inb && ra != repb && linked_if(near, x, qb, g);
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
// its members are friends): first the 3 forward face offsets of every
// non-empty sub-cell, then the other 118 offsets of the 5x5x5 stencil from
// the sub-cells outside the largest component, each round over the
// (sub-cell, non-empty neighbour) tasks spread over the lanes; finally
// parent[slot] = first slot of the slot's local component.
constexpr int kDenseWarps = 4;  // default warps per CTA (the autotuner may pick 8)

__device__ __forceinline__ int sub_key(float4 q, const LinkGeom &g, int cx, int cy, int cz) {
    return sub_coord(q.x, g.inv_fine, cx, g.k) +
           g.k * (sub_coord(q.y, g.inv_fine, cy, g.k) + g.k * sub_coord(q.z, g.inv_fine, cz, g.k));
}

// One round of the dense-cell local union-find over (source sub-cell F,
// offset) tasks whose sub-cell G = F + offset is non-empty.  The candidate
// offsets of F come from the occupancy rows (bit x of rows[z*k + y] = sub-cell
// (x, y, z) non-empty), read a row of five offsets at a time; the tasks of 32
// sources are laid out in shared memory (a window of tcap at a time) and then
// taken by the lanes in turn, so no lane idles on an empty neighbour.  A task
// is skipped when F and G are already in one component, else the pair of
// sub-cells is tested until its first link.  Offset sets (MODE):
//   kFace  the 3 forward face offsets (+x, +y, +z)
//   kRest  the other 118 offsets of the 5x5x5 stencil, both directions
constexpr int kFace = 0, kRest = 1;

template <int MODE>
__device__ __forceinline__ uint32_t row_bits(const uint32_t *rows, int k, int x, int yy, int zz, int dy, int dz) {
    if (unsigned(yy) >= unsigned(k) || unsigned(zz) >= unsigned(k)) return 0u;
    uint32_t w = ((rows[zz * k + yy] << 2) >> x) & 31u;  // bit dx + 2 for dx in [-2, 2]
    int ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
    uint32_t allow;
    if (MODE == kFace)
        allow = (ay + az == 0) ? 0x08u : 0x04u;
    else if (ay == 2 || az == 2)
        allow = 0x1Fu;  // a component of +-2: all five
    else if (ay + az == 0)
        allow = 0x11u;  // dx = +-2 (+-1 are faces, 0 is the sub-cell itself)
    else if (ay + az == 1)
        allow = 0x1Bu;  // dx = 0 is a face
    else
        allow = 0x1Fu;  // edges and corners
    return w & allow;
}

// Visits the candidate rows of a source: f(dy, dz, bits).
template <int MODE, class Fn>
__device__ __forceinline__ void for_rows(const uint32_t *rows, int k, int x, int y, int z, Fn f) {
    if (MODE == kFace) {
        f(0, 0, row_bits<kFace>(rows, k, x, y, z, 0, 0));
        f(1, 0, row_bits<kFace>(rows, k, x, y + 1, z, 1, 0));
        f(0, 1, row_bits<kFace>(rows, k, x, y, z + 1, 0, 1));
    } else {
#pragma unroll 1
        for (int dz = -2; dz <= 2; ++dz)
#pragma unroll
            for (int dy = -2; dy <= 2; ++dy) f(dy, dz, row_bits<kRest>(rows, k, x, y + dy, z + dz, dy, dz));
    }
}

template <int MODE>
__device__ void dense_round(const uint32_t *src, int nsrc, int k, const uint16_t *ss, int *lp,
                            const float4 *__restrict__ cp, const LinkGeom &g, int lane, const uint32_t *rows,
                            uint32_t *tasks, int tcap) {
    for (int b0 = 0; b0 < nsrc; b0 += 32) {
        const int i = b0 + lane;
        const uint32_t e = i < nsrc ? src[i] : 0u;  // key | x << 10 | y << 14 | z << 18
        const int F = int(e & 1023u), x = int((e >> 10) & 15u), y = int((e >> 14) & 15u), z = int((e >> 18) & 15u);
        int c = 0;
        if (i < nsrc) for_rows<MODE>(rows, k, x, y, z, [&](int, int, uint32_t bits) { c += __popc(bits); });
        int pre = c;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31);
        pre -= c;
        for (int w0 = 0; w0 < total; w0 += tcap) {
            if (i < nsrc && c > 0 && pre < w0 + tcap && pre + c > w0) {
                int idx = pre;
                for_rows<MODE>(rows, k, x, y, z, [&](int dy, int dz, uint32_t bits) {
                    while (bits) {
                        int b = __ffs(int(bits)) - 1;
                        bits &= bits - 1u;
                        if (idx >= w0 && idx < w0 + tcap) {
                            int G = F + (b - 2) + k * (dy + k * dz);
                            tasks[idx - w0] = uint32_t(F) | uint32_t(G) << 16;
                        }
                        ++idx;
                    }
                });
            }
            __syncwarp();
            const int nt = min(tcap, total - w0);
            for (int t = lane; t < nt; t += 32) {
                uint32_t tk = tasks[t];
                int Fs = int(tk & 0xFFFFu), G = int(tk >> 16);
                if (lfind(lp, Fs) == lfind(lp, G)) continue;
                int f0 = ss[Fs], f1 = ss[Fs + 1], g0 = ss[G], g1 = ss[G + 1];
                bool done = false;
                for (int a = f0; a < f1 && !done; ++a) {
                    float4 pa = cp[a];
                    for (int cc = g0; cc < g1; ++cc) {
                        if (linked_near(pa, cp[cc], g)) {  // one cell, n >= 5
                            lunite(lp, Fs, G);
                            done = true;
                            break;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

template <int W>
__global__ void __launch_bounds__(32 * W) dense_cells_kernel(float4 *__restrict__ spos,
                                                                       float4 *__restrict__ stage,
                                                                       const uint32_t *__restrict__ cell_start,
                                                                       const uint32_t *__restrict__ dense_cells,
                                                                       const uint32_t *__restrict__ ndense,
                                                                       uint32_t *next, uint16_t *__restrict__ sub_start,
                                                                       uint16_t *__restrict__ sub_rows,
                                                                       int *__restrict__ parent, LinkGeom g) {
    __shared__ int sh_cnt[W][kSubMax + 1];
    __shared__ uint16_t sh_ss[W][kSubMax + 2];
    __shared__ uint32_t sh_ne[W][kSubMax + 1];
    __shared__ int sh_sz[W][kSubMax + 1];
    __shared__ uint32_t sh_rows[W][kSubSide * kSubSide];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *cnt = sh_cnt[w];
    uint16_t *ss = sh_ss[w];
    uint32_t *ne = sh_ne[w];
    int *sz = sh_sz[w];
    uint32_t *rows = sh_rows[w];
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
        for (int r = lane; r < k * k; r += 32) rows[r] = 0u;
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
                atomicOr(&rows[ky + k * kz], 1u << kx);
            }
            pre += c;
        }
        if (lane == 0) {
            ss[k3] = uint16_t(m);
            tab[k3] = uint16_t(m);
        }
        __syncwarp();
        for (int r = lane; r < k * k; r += 32) sub_rows[d * (kSubSide * kSubSide) + r] = uint16_t(rows[r]);
        for (int t = lane; t < m; t += 32) {
            float4 q = stage[start + t];
            int r = atomicAdd(&cnt[sub_key(q, g, cx, cy, cz)], 1);
            spos[start + r] = q;
        }
        __syncwarp();
        for (int key = lane; key < k3; key += 32) cnt[key] = key;
        __syncwarp();
        dense_round<kFace>(ne, nF, k, ss, cnt, spos + start, g, lane, rows, reinterpret_cast<uint32_t *>(sz),
                          kSubMax + 1);
        __syncwarp();
        // full compression: every sub-cell points at its root, so the finds of
        // the second round are one load deep
        for (int i = lane; i < nF; i += 32) cnt[ne[i] & 1023u] = lfind(cnt, int(ne[i] & 1023u));
        __syncwarp();
        // The second round (every offset but the faces) can only join sub-cells
        // still in different components.  Every such pair has an end outside
        // the largest component, so the round runs only from the sub-cells
        // outside it, over those offsets in both directions.
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
        if (nmin > 0) dense_round<kRest>(minority, nmin, k, ss, cnt, spos + start, g, lane, rows, ne, kSubMax + 1);
        __syncwarp();
        for (int t = lane; t < m; t += 32) {
            float4 q = spos[start + t];
            parent[start + t] = int(start) + ss[lfind(cnt, sub_key(q, g, cx, cy, cz))];
        }
        __syncwarp();
    }
}

// Non-empty sub-cells of a dense cell (occupancy rows) inside box b: f(G)
// for each, in a fixed order.
template <class Fn>
__device__ __forceinline__ void for_box(const uint16_t *rows, int k, SubBox b, Fn f) {
    const uint32_t xm = (1u << (b.x1 - b.x0 + 1)) - 1u;
    for (int z = b.z0; z <= b.z1; ++z)
        for (int y = b.y0; y <= b.y1; ++y) {
            uint32_t bits = (uint32_t(rows[z * k + y]) >> b.x0) & xm;
            while (bits) {
                int i = __ffs(int(bits)) - 1;
                bits &= bits - 1u;
                f(b.x0 + i + k * (y + k * z));
            }
        }
}

__device__ __forceinline__ int box_count(const uint16_t *rows, int k, SubBox b) {
    const uint32_t xm = (1u << (b.x1 - b.x0 + 1)) - 1u;
    int c = 0;
    for (int z = b.z0; z <= b.z1; ++z)
        for (int y = b.y0; y <= b.y1; ++y) c += __popc((uint32_t(rows[z * k + y]) >> b.x0) & xm);
    return c;
}

// Box within 2 sub-cells of position (cx, cy, cz) (may lie outside the cell),
// clipped to the cell; false when empty.
__device__ __forceinline__ bool near_box(int cx, int cy, int cz, int k, SubBox &b) {
    b.x0 = max(cx - 2, 0);
    b.y0 = max(cy - 2, 0);
    b.z0 = max(cz - 2, 0);
    b.x1 = min(cx + 2, k - 1);
    b.y1 = min(cy + 2, k - 1);
    b.z1 = min(cz + 2, k - 1);
    return b.x0 <= b.x1 && b.y0 <= b.y1 && b.z0 <= b.z1;
}

// Dense cells, part 2: one warp per dense cell A, its pairs with neighbours.
//   small / medium neighbour B (any direction): each particle q of B within
//   reach of A is paired with the non-empty sub-cells of A within 2 sub-cells
//   of q's position
//   dense forward neighbour B: each non-empty sub-cell F of A in the two
//   layers facing B is paired with the non-empty sub-cells of B within 2
//   sub-cells of F
// The (source, sub-cell) tasks come from the occupancy rows of the two cells
// and are spread over the lanes; a task is skipped when its two ends are
// already in one component, else tested until the first link.
constexpr int kNbrWarps = 8;  // default warps per CTA (the autotuner may pick 4)
constexpr int kNbrTaskCap = 512;
constexpr int kNbrSrcCap = 2 * kSubSide * kSubSide;

template <int W>
__global__ void __launch_bounds__(32 * W) dense_nbr_kernel(const float4 *__restrict__ spos,
                                                                   const uint32_t *__restrict__ cell_start,
                                                                   const uint32_t *__restrict__ dense_cells,
                                                                   const uint32_t *__restrict__ ndense, uint32_t *next,
                                                                   const uint32_t *__restrict__ dense_id,
                                                                   const uint16_t *__restrict__ sub_start,
                                                                   const uint16_t *__restrict__ sub_rows, LinkGeom g,
                                                                   int *parent, DevStatus st) {
    __shared__ uint32_t sh_task[W][kNbrTaskCap];
    __shared__ uint32_t sh_src[W][kNbrSrcCap];
    __shared__ float4 sh_q[W][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *tasks = sh_task[w];
    uint32_t *srcl = sh_src[w];
    float4 *qbuf = sh_q[w];
    int64_t D = *ndense;
    if (D > g.D_cap) D = g.D_cap;
    const int k = g.k, kk = k * k;
    for (int64_t d = next_task(next, lane); d < D; d = next_task(next, lane)) {
        if (g.n < 3) break;
        uint32_t ga = dense_cells[d];
        int cx, cy, cz;
        decode_cell(ga, g.nb, cx, cy, cz);
        const bool near = interior_cell(cx, cy, cz, g);
        const uint32_t a0 = cell_start[ga];
        const uint16_t *ta = sub_start + d * (kSubMax + 1);
        const uint16_t *ra = sub_rows + d * (kSubSide * kSubSide);
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
            const uint32_t b0 = __shfl_sync(0xffffffffu, nb0, o), b1 = __shfl_sync(0xffffffffu, nb1, o);
            const int off[3] = {c_nb26[o][0], c_nb26[o][1], c_nb26[o][2]};
            const int bx = wrapc(cx + off[0], g.n), by = wrapc(cy + off[1], g.n), bz = wrapc(cz + off[2], g.n);
            if (cls != 3) {
                const int mB = int(b1 - b0);
                for (int cb = 0; cb < mB; cb += 32) {
                    const int j = cb + lane;
                    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool inb = j < mB;
                    SubBox bx3{0, 0, 0, -1, -1, -1};
                    if (inb) {
                        q = spos[b0 + j];
                        inb = gap_to_neighbour(q, bx, by, bz, -off[0], -off[1], -off[2], g.cell_side) <= g.gap2;
                    }
                    if (inb) {
                        // q's sub-cell in A's frame, and the box of A's sub-cells within 2 of it
                        inb = near_box(sub_coord(q.x, g.inv_fine, bx, k) + off[0] * k,
                                       sub_coord(q.y, g.inv_fine, by, k) + off[1] * k,
                                       sub_coord(q.z, g.inv_fine, bz, k) + off[2] * k, k, bx3);
                    }
                    if (!__any_sync(0xffffffffu, inb)) continue;
                    qbuf[lane] = q;
                    const int c = inb ? box_count(ra, k, bx3) : 0;
                    __syncwarp();
                    warp_tasks(
                        c, tasks, kNbrTaskCap, lane,
                        [&](auto put) { for_box(ra, k, bx3, [&](int G) { put(uint32_t(lane) | uint32_t(G) << 5); }); },
                        [&](uint32_t t) {
                            const int qi = int(t & 31u), G = int(t >> 5);
                            const int qs = int(b0) + cb + qi;
                            const uint32_t c0 = ta[G], c1 = ta[G + 1];
                            if (uf_find(parent, qs) == uf_find(parent, int(a0 + c0))) return;
                            const float4 qq = qbuf[qi];
                            for (uint32_t cc = c0; cc < c1; ++cc)
                                if (linked_if(near, qq, spos[a0 + cc], g)) {
                                    uf_unite(parent, qs, int(a0 + cc), st);
                                    break;
                                }
                        });
                }
                continue;
            }
            const int64_t db = int64_t(__shfl_sync(0xffffffffu, nid, o));
            const uint16_t *tb = sub_start + db * (kSubMax + 1);
            const uint16_t *rb = sub_rows + db * (kSubSide * kSubSide);
            // sources: the non-empty sub-cells of A in the two layers facing B
            int slo[3], shi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                slo[a] = off[a] > 0 ? k - 2 : 0;
                shi[a] = off[a] < 0 ? 1 : k - 1;
            }
            int nsrc = 0;
            for (int r0 = 0; r0 < kk; r0 += 32) {
                const int r = r0 + lane;
                const int y = r % k, z = r / k;
                uint32_t bits = 0u;
                if (r < kk && y >= slo[1] && y <= shi[1] && z >= slo[2] && z <= shi[2])
                    bits = (uint32_t(ra[r]) >> slo[0]) & ((1u << (shi[0] - slo[0] + 1)) - 1u);
                int c = __popc(bits), pre = c;
                for (int sh = 1; sh < 32; sh <<= 1) {
                    int v = __shfl_up_sync(0xffffffffu, pre, sh);
                    if (lane >= sh) pre += v;
                }
                int idx = nsrc + pre - c;
                while (bits) {
                    int b = __ffs(int(bits)) - 1;
                    bits &= bits - 1u;
                    int x = slo[0] + b;
                    srcl[idx++] = uint32_t(x) | uint32_t(y) << 4 | uint32_t(z) << 8;
                }
                nsrc += __shfl_sync(0xffffffffu, pre, 31);
            }
            __syncwarp();
            for (int s0 = 0; s0 < nsrc; s0 += 32) {
                const int i = s0 + lane;
                int F = 0;
                SubBox fb3{0, 0, 0, -1, -1, -1};
                bool has = i < nsrc;
                if (has) {
                    uint32_t e = srcl[i];
                    int fx = int(e & 15u), fy = int((e >> 4) & 15u), fz = int((e >> 8) & 15u);
                    F = fx + k * (fy + k * fz);
                    // F's position in B's frame, and B's sub-cells within 2 of it
                    has = near_box(fx - off[0] * k, fy - off[1] * k, fz - off[2] * k, k, fb3);
                }
                const int c = has ? box_count(rb, k, fb3) : 0;
                warp_tasks(
                    c, tasks, kNbrTaskCap, lane,
                    [&](auto put) { for_box(rb, k, fb3, [&](int G) { put(uint32_t(F) | uint32_t(G) << 16); }); },
                    [&](uint32_t t) {
                        const int Fs = int(t & 0xFFFFu), G = int(t >> 16);
                        const uint32_t f0 = ta[Fs], f1 = ta[Fs + 1], c0 = tb[G], c1 = tb[G + 1];
                        if (uf_find(parent, int(a0 + f0)) == uf_find(parent, int(b0 + c0))) return;
                        bool done = false;
                        for (uint32_t a = f0; a < f1 && !done; ++a) {
                            const float4 p = spos[a0 + a];
                            for (uint32_t cc = c0; cc < c1; ++cc)
                                if (linked_if(near, p, spos[b0 + cc], g)) {
                                    uf_unite(parent, int(a0 + a), int(b0 + cc), st);
                                    done = true;
                                    break;
                                }
                        }
                    });
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
LinkParams make_link_params(int64_t N, float L, float b, int n, int S, int T, int shape) {
    LinkParams lp{};
    if (T < 0) T = default_dense_threshold(N);
    const int w[3][4] = {{kMedWarps, kMedXWarps, kDenseWarps, kNbrWarps}, {8, 8, 8, 8}, {4, 4, 4, 4}};
    const int sh = shape >= 0 && shape < kCtaShapes ? shape : 0;
    for (int q = 0; q < 4; ++q) lp.warps[q] = w[sh][q];
    double s = double(L) / n;
    int k = int(std::ceil(s * std::sqrt(3.0) * 1.02 / double(b)));
    if (k < 1) k = 1;
    double sf = s / k;
    double eps = 4.0 * double(L) * std::ldexp(1.0, -24);
    bool ok = T > 0 && n >= 5 && k <= kSubSide && std::sqrt(3.0) * (sf + 2 * eps) <= double(b) * (1 - 1e-4) &&
              (double(b) + 2 * eps) / sf < 2.0;
    lp.S = S < 0 ? 0 : (S > kSmallMax ? kSmallMax : S);
    lp.T = ok ? (T > lp.S ? T : lp.S + 1) : 0;
    lp.k = k;
    lp.inv_fine = float(double(n) * k / double(L));
    lp.D_cap = ok ? dense_cap(N) : 0;
    return lp;
}

void launch_link_core(const jfof_cells &c, const FofBuffers &fb, const LinkParams &lp, const DevStatus &st,
                      cudaStream_t s) {
    int64_t N = c.n;
    float b2 = host_mul(c.b, c.b);
    double gap = 1.02 * double(c.b);
    LinkGeom g{c.L, 0.5f * c.L, b2, float(double(c.n_axis) / double(c.L)), lp.inv_fine,
               float(double(c.L) / c.n_axis), float(gap * gap), c.n_axis, bricks_per_axis(c.n_axis), lp.k,
               lp.k * lp.k * lp.k, lp.S, lp.T, lp.D_cap};
    const float4 *spos = reinterpret_cast<const float4 *>(c.spos);
    // Warps of the list-driven kernels (they take cells from a work counter, so
    // any count is correct): at most one per cell the class can hold, so a
    // small box does not launch a full grid of warps that find no work.
    auto list_threads = [&](int64_t cap, int64_t min_particles) {
        int64_t w = N / min_particles + 1;
        return (w < cap ? w : cap) * 32;
    };
    const int64_t med_thr = list_threads(medium_cap(N), lp.S + 1), dense_thr = list_threads(lp.D_cap, lp.T + 1);
    const int64_t big_thr = list_threads(medium_cap(N), kMedMain + 1);
    {
        JFOF_TRACE("link_init", s);
        iota_kernel<<<grid_for(N, 256), 256, 0, s>>>(fb.parent, N);
    }
    cudaMemsetAsync(fb.counters + 2, 0, 4 * sizeof(uint32_t), s);  // work counters
    cudaMemsetAsync(fb.counters + 7, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(fb.counters + 9, 0, 2 * sizeof(uint32_t), s);
    // local passes first: they write parent with plain stores, each for its own cell
    if (lp.T > 0) {
        JFOF_TRACE("dense_cells", s);
        auto k = lp.warps[2] == 8 ? dense_cells_kernel<8> : dense_cells_kernel<4>;
        k<<<grid_for(dense_thr, 32 * lp.warps[2], 8), 32 * lp.warps[2], 0, s>>>(
            fb.spos, fb.tmp, c.cell_start, fb.dense_cells, fb.counters, fb.counters + 2, fb.sub_start, fb.sub_rows,
            fb.parent, g);
    }
    {
        JFOF_TRACE("link_medium_local", s);
        // pairs of one cell need no minimum image once cells are at most L/3 wide
        const bool W8 = lp.warps[0] == 8, nr = c.n_axis >= 3;
        auto k = nr ? (W8 ? medium_local_kernel<8, true, false> : medium_local_kernel<4, true, false>)
                    : (W8 ? medium_local_kernel<8, false, false> : medium_local_kernel<4, false, false>);
        k<<<grid_for(med_thr, 32 * lp.warps[0], 8), 32 * lp.warps[0], 0, s>>>(
            spos, c.cell_start, fb.medium_cells, fb.counters + 1, fb.counters + 3, medium_cap(N), g, fb.parent, st);
        auto kb = nr ? (W8 ? medium_local_kernel<8, true, true> : medium_local_kernel<4, true, true>)
                     : (W8 ? medium_local_kernel<8, false, true> : medium_local_kernel<4, false, true>);
        kb<<<grid_for(big_thr, 32 * lp.warps[0], 8), 32 * lp.warps[0], 0, s>>>(
            spos, c.cell_start, fb.medium_cells, fb.counters + 8, fb.counters + 9, medium_cap(N), g, fb.parent, st);
    }
    // then everything that unites across cells (atomic hooks only)
    if (lp.S > 0) {
        JFOF_TRACE("link_small", s);
        small_kernel<<<grid_for(N, 32 * kSmallWarps, 8), 32 * kSmallWarps, 0, s>>>(spos, c.cell_start, fb.small_slots, fb.counters + 6,
                                                          fb.counters + 7, g, fb.parent, st);
    }
    {
        JFOF_TRACE("link_medium", s);
        auto k = lp.warps[1] == 4 ? medium_kernel<4, false> : medium_kernel<8, false>;
        k<<<grid_for(med_thr, 32 * lp.warps[1], 8), 32 * lp.warps[1], 0, s>>>(
            spos, c.cell_start, fb.medium_cells, fb.counters + 1, fb.counters + 4, fb.dense_id, medium_cap(N), g,
            fb.parent, st);
        auto kb = lp.warps[1] == 4 ? medium_kernel<4, true> : medium_kernel<8, true>;
        kb<<<grid_for(big_thr, 32 * lp.warps[1], 8), 32 * lp.warps[1], 0, s>>>(
            spos, c.cell_start, fb.medium_cells, fb.counters + 8, fb.counters + 10, fb.dense_id, medium_cap(N), g,
            fb.parent, st);
    }
    if (lp.T > 0) {
        JFOF_TRACE("link_dense_nbr", s);
        auto k = lp.warps[3] == 4 ? dense_nbr_kernel<4> : dense_nbr_kernel<8>;
        k<<<grid_for(dense_thr, 32 * lp.warps[3], 8), 32 * lp.warps[3], 0, s>>>(
            spos, c.cell_start, fb.dense_cells, fb.counters, fb.counters + 5, fb.dense_id, fb.sub_start, fb.sub_rows,
            g, fb.parent, st);
    }
}

void launch_link(const jfof_cells &c, const FofBuffers &fb, const LinkParams &lp, int32_t *label,
                 const DevStatus &st, cudaStream_t s) {
    launch_link_core(c, fb, lp, st, s);
    launch_tail_labels(fb, c.n, label, s);
}

}  // namespace jfof
