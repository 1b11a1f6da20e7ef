// k_reinforce.cu -- a11-a13: the REINFORCE topological mode (Sec. 3.2).
//
//   a11  fixed candidate list (the neighbour list is not rebuilt, Sec. 3.2):
//        unordered pairs i < j with d2 < r_cut^2, sorted by (i, j), with the
//        distance d and the edge probability p (Eq. 8 or the distance sigmoid)
//   a12  K samples: edge (i, j) present in sample k iff u < p, u from
//        Philox4x32-10 (Salmon et al., SC'11) keyed by the seed at counter
//        (min, max, floor(k/4), 0), word k mod 4, top 24 bits; per-sample FoF
//        labels (smallest member index) and halo counts
//   a13  score-function gradient (Eqs. 6-7): g = (1/K) sum_k A_k dlog p(y_k)/dx
//        with dlog p/dz_e = y_e - p_e and z_e's derivative in positions;
//        deterministic per-particle sums over a fixed pair order
#include "jfof_internal.cuh"
#include "k_fof.cuh"
#include "k_reinforce.cuh"

namespace jfof {

// ---------------------------------------------------------------------------
// Binary32 exponential: Cody-Waite reduction x = k ln2 + r with ln2 split in
// a binary32 head and tail, the degree-7 Taylor polynomial sum r^m/m! by
// Horner with fused multiply-add, and scaling by 2^k through the exponent
// field; input clamped to [-87, 87].  Constants: 1/ln2, ln2 and the remainder
// ln2 - f32(ln2), and 1/m! (m = 0..7), each rounded once to binary32.
__device__ __forceinline__ float jexp(float x) {
    const float l2e = __uint_as_float(0x3FB8AA3Bu);
    const float ln2_hi = __uint_as_float(0x3F317218u);
    const float ln2_lo = __uint_as_float(0xB102E308u);
    if (x != x) x = 0.0f;
    x = fminf(fmaxf(x, -87.0f), 87.0f);
    float k = rintf(__fmul_rn(x, l2e));
    float r = __fmaf_rn(-k, ln2_hi, x);
    r = __fmaf_rn(-k, ln2_lo, r);
    float p = __uint_as_float(0x39500D01u);               // 1/7!
    p = __fmaf_rn(p, r, __uint_as_float(0x3AB60B61u));    // 1/6!
    p = __fmaf_rn(p, r, __uint_as_float(0x3C088889u));    // 1/5!
    p = __fmaf_rn(p, r, __uint_as_float(0x3D2AAAABu));    // 1/4!
    p = __fmaf_rn(p, r, __uint_as_float(0x3E2AAAABu));    // 1/3!
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    float scale = __int_as_float((int(k) + 127) << 23);
    return __fmul_rn(p, scale);
}

__device__ __forceinline__ float edge_prob(float d, float d2, float b, float b2, int form, float coef) {
    float z = form == 0 ? __fmul_rn(__fsub_rn(b, d), coef) : __fmul_rn(__fsub_rn(b2, d2), coef);
    return __fdiv_rn(1.0f, __fadd_rn(1.0f, jexp(-z)));
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 edge_words(uint64_t seed, int i, int j, int group) {
    uint32_t lo = uint32_t(min(i, j)), hi = uint32_t(max(i, j));
    return philox4x32_10(make_uint4(lo, hi, uint32_t(group), 0u), make_uint2(uint32_t(seed), uint32_t(seed >> 32)));
}

__device__ __forceinline__ float word_uniform(uint32_t w) { return __fmul_rn(float(w >> 8), 5.9604644775390625e-8f); }

__device__ __forceinline__ uint32_t pick(uint4 v, int w) { return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w)); }

// ---------------------------------------------------------------------------
// a11: the candidate list.  One thread per particle (sorted order) scans the
// 27 cells of a grid with cells >= 1.01 r_cut; counts, then fills, partners
// j > i (original indices), which a segmented sort puts in ascending order.
__global__ void __launch_bounds__(256) pair_scan_kernel(const float4 *__restrict__ spos,
                                                        const uint32_t *__restrict__ cell_start, int64_t N, PairGeom g,
                                                        uint32_t *__restrict__ cnt, const uint32_t *__restrict__ off,
                                                        int64_t cap, int32_t *__restrict__ pair_i,
                                                        int32_t *__restrict__ pair_j,
                                                        unsigned long long *__restrict__ total) {
    const bool fill = off != nullptr;
    if (fill && uint64_t(off[N]) > uint64_t(cap)) return;
    uint32_t local = 0;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        float4 p = spos[s];
        int i = __float_as_int(p.w);
        int cx = cell_coord(p.x, g.inv_cell, g.n), cy = cell_coord(p.y, g.inv_cell, g.n),
            cz = cell_coord(p.z, g.inv_cell, g.n);
        uint32_t c = 0, w0 = fill ? off[i] : 0;
        int reach = g.n >= 3 ? 1 : 0;
        for (int dz = -reach; dz <= reach; ++dz)
            for (int dy = -reach; dy <= reach; ++dy)
                for (int dx = -reach; dx <= reach; ++dx) {
                    int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                    nx = nx < 0 ? nx + g.n : (nx >= g.n ? nx - g.n : nx);
                    ny = ny < 0 ? ny + g.n : (ny >= g.n ? ny - g.n : ny);
                    nz = nz < 0 ? nz + g.n : (nz >= g.n ? nz - g.n : nz);
                    uint64_t cell = cell_table_index(nx, ny, nz, g.nb);
                    uint32_t b0 = cell_start[cell], b1 = cell_start[cell + 1];
                    for (uint32_t t = b0; t < b1; ++t) {
                        float4 q = spos[t];
                        int j = __float_as_int(q.w);
                        if (j <= i || !(pair_d2(p, q, g.L, g.hL) < g.rc2)) continue;
                        if (fill) {
                            pair_i[w0 + c] = i;
                            pair_j[w0 + c] = j;
                        }
                        ++c;
                    }
                }
        if (!fill) cnt[i] = c;
        local += c;
    }
    if (!fill) {
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, (unsigned long long)local);
    }
}

__global__ void __launch_bounds__(256) pair_props_kernel(const float *__restrict__ pos, PairGeom g,
                                                         const uint32_t *__restrict__ off, int64_t N, int64_t cap,
                                                         const int32_t *__restrict__ pair_i,
                                                         const int32_t *__restrict__ pair_j, float *__restrict__ pair_d,
                                                         float *__restrict__ pair_p) {
    int64_t E = off[N];
    if (E > cap) return;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
        int i = pair_i[e], j = pair_j[e];
        float4 p, q;
        float a[3], c[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            a[t] = pos[3 * int64_t(i) + t];
            c[t] = pos[3 * int64_t(j) + t];
            if (g.wrap) {
                a[t] = wrap_coord(a[t], g.L);
                c[t] = wrap_coord(c[t], g.L);
            }
        }
        p = make_float4(a[0], a[1], a[2], 0.f);
        q = make_float4(c[0], c[1], c[2], 0.f);
        float d2 = pair_d2(p, q, g.L, g.hL);
        float d = __fsqrt_rn(d2);
        pair_d[e] = d;
        pair_p[e] = edge_prob(d, d2, g.b, g.b2, g.form, g.coef);
    }
}

__global__ void pair_total_kernel(const uint32_t *off, int64_t N, const unsigned long long *total, int64_t cap,
                                  int64_t *n_pairs, DevStatus st) {
    unsigned long long t = *total;
    *n_pairs = int64_t(t);
    if (t > 0xffffffffull) latch(st, JFOF_EOVERFLOW);
    else if (int64_t(t) > cap && cap > 0) latch(st, JFOF_EOVERFLOW);
    (void)off;
    (void)N;
}

struct LoadCnt {
    const uint32_t *p;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return p[i]; }
};

size_t pairs_layout(int64_t N, int n, PairBuffers *pb, void *base) {
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    PairBuffers b;
    b.cnt = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N)));
    b.off = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N + 1)));
    b.scan_tmp = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * scan_tmp_words(N)));
    b.total = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long)));
    b.seglist_words = segsort_list_words(N);
    b.seglist = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(b.seglist_words)));
    b.cells_ws = take(fof_layout(N, n, nullptr, nullptr));
    if (pb) *pb = b;
    return off;
}

void launch_pairs(const float *pos, int64_t N, const PairGeom &pg, const PairBuffers &pb, int64_t cap,
                  int32_t *pair_i, int32_t *pair_j, float *pair_d, float *pair_p, int64_t *n_pairs,
                  const DevStatus &st, cudaStream_t s) {
    FofBuffers fb;
    fof_layout(N, pg.n, &fb, pb.cells_ws);
    LinkParams lp{};
    lp.S = INT32_MAX;  // no class lists needed
    launch_bin_cells(pos, N, pg.L, pg.n, pg.wrap, lp, fb, st, s);
    cudaMemsetAsync(pb.total, 0, sizeof(unsigned long long), s);
    {
        JFOF_TRACE("pair_count", s);
        pair_scan_kernel<<<grid_for(N, 256), 256, 0, s>>>(fb.spos, fb.cell_start, N, pg, pb.cnt, nullptr, cap,
                                                          nullptr, nullptr, pb.total);
    }
    {
        JFOF_TRACE("scan", s);
        scan_exclusive(LoadCnt{pb.cnt}, N, pb.off, pb.scan_tmp, s);
    }
    pair_total_kernel<<<1, 1, 0, s>>>(pb.off, N, pb.total, cap, n_pairs, st);
    if (cap <= 0) return;
    {
        JFOF_TRACE("pair_fill", s);
        pair_scan_kernel<<<grid_for(N, 256), 256, 0, s>>>(fb.spos, fb.cell_start, N, pg, pb.cnt, pb.off, cap,
                                                          pair_i, pair_j, pb.total);
    }
    // every segment holds pairs (i, j) of one i: sort j ascending (pair_i is constant there)
    launch_segsort(pb.off, N, pair_j, cap, s, nullptr, pb.seglist, pb.seglist_words);
    {
        JFOF_TRACE("pair_props", s);
        pair_props_kernel<<<grid_for(N * 16, 256), 256, 0, s>>>(pos, pg, pb.off, N, cap, pair_i, pair_j, pair_d,
                                                                pair_p);
    }
}

// ---------------------------------------------------------------------------
// a12: per-sample FoF over the sampled edges.  labels[k] doubles as the
// union-find forest of sample k (root = smallest index).  Samples run in
// chunks of 16 so the chunk's forests stay in L2.
__global__ void rows_iota_kernel(int32_t *__restrict__ rows, int64_t N, int nrows) {
    int64_t total = N * nrows;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x)
        rows[t] = int32_t(t % N);
}

// blockIdx.y = group of four samples within the chunk
__global__ void __launch_bounds__(256) sample_union_kernel(const int32_t *__restrict__ pair_i,
                                                           const int32_t *__restrict__ pair_j,
                                                           const float *__restrict__ pair_p, int64_t E, int64_t N,
                                                           int k0, int kc, int K, uint64_t seed, int32_t *labels,
                                                           DevStatus st) {
    int gk = k0 / 4 + int(blockIdx.y);  // global group index
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
        int i = pair_i[e], j = pair_j[e];
        float p = pair_p[e];
        uint4 u4 = edge_words(seed, i, j, gk);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            int k = 4 * gk + w;
            if (k < k0 || k >= k0 + kc || k >= K) continue;
            if (word_uniform(pick(u4, w)) < p) uf_unite(labels + int64_t(k) * N, i, j, st);
        }
    }
}

__global__ void __launch_bounds__(256) rows_finalize_kernel(int32_t *rows, int64_t N, int nrows,
                                                            uint32_t *__restrict__ counts) {
    int64_t total = N * nrows;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        int64_t r = t / N, i = t - r * N;
        int32_t *row = rows + r * N;
        int root = uf_find_ro(row, int(i));
        row[i] = root;
        atomicAdd(&counts[r * N + root], 1u);
    }
}

__global__ void __launch_bounds__(256) rows_halos_kernel(const int32_t *__restrict__ rows, int64_t N, int nrows,
                                                         const uint32_t *__restrict__ counts, uint32_t min_size,
                                                         int32_t *__restrict__ n_halos) {
    int64_t total = N * nrows;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        int64_t r = t / N, i = t - r * N;
        if (rows[t] == int32_t(i) && counts[t] >= min_size) atomicAdd(&n_halos[r], 1);
    }
}

size_t sample_layout(int64_t N, uint32_t **counts, void *base) {
    size_t bytes = align_up(sizeof(uint32_t) * size_t(N) * kSampleChunk);
    if (counts) *counts = reinterpret_cast<uint32_t *>(base);
    return bytes;
}

void launch_reinforce_sample(int64_t N, const int32_t *pair_i, const int32_t *pair_j, const float *pair_p, int64_t E,
                             int32_t K, uint64_t seed, int32_t min_size, uint32_t *counts, int32_t *labels,
                             int32_t *n_halos, const DevStatus &st, cudaStream_t s) {
    cudaMemsetAsync(n_halos, 0, sizeof(int32_t) * size_t(K), s);
    for (int k0 = 0; k0 < K; k0 += kSampleChunk) {
        int kc = K - k0 < kSampleChunk ? K - k0 : kSampleChunk;
        int32_t *rows = labels + int64_t(k0) * N;
        {
            JFOF_TRACE("sample_init", s);
            rows_iota_kernel<<<grid_for(N * kc, 256), 256, 0, s>>>(rows, N, kc);
        }
        if (E > 0) {
            JFOF_TRACE("sample_union", s);
            dim3 grid(unsigned(grid_for(E, 256, 2)), unsigned((kc + 3) / 4));
            sample_union_kernel<<<grid, 256, 0, s>>>(pair_i, pair_j, pair_p, E, N, k0, kc, K, seed, labels, st);
        }
        cudaMemsetAsync(counts, 0, sizeof(uint32_t) * size_t(N) * kc, s);
        {
            JFOF_TRACE("sample_finalize", s);
            rows_finalize_kernel<<<grid_for(N * kc, 256), 256, 0, s>>>(rows, N, kc, counts);
        }
        {
            JFOF_TRACE("sample_halos", s);
            rows_halos_kernel<<<grid_for(N * kc, 256), 256, 0, s>>>(rows, N, kc, counts, uint32_t(min_size),
                                                                    n_halos + k0);
        }
    }
}

// ---------------------------------------------------------------------------
// a13: score-function gradient.
//   c_e = (1/K) (sum_k A_k y_ke - p_e sum_k A_k)          (Kahan, binary32)
//   form 0: dz/dx_i = (x_j - x_i)_mi / (tau d)  -> fac = (1/tau)/d  (0 if d = 0)
//   form 1: dz/dx_i = 2 (alpha/b2) (x_j - x_i)_mi -> fac = 2 alpha/b2
//   g_i += c_e fac (x_j - x_i)_mi,  g_j -= the same.
// Each particle sums its pairs in a fixed order: first those where it is i
// (ascending j), then those where it is j (ascending pair index).
__global__ void sum_adv_kernel(const float *adv, int K, float *sumA) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f, c = 0.f;
        for (int k = 0; k < K; ++k) {
            float y = __fsub_rn(adv[k], c), t = __fadd_rn(s, y);
            c = __fsub_rn(__fsub_rn(t, s), y);
            s = t;
        }
        *sumA = __fsub_rn(s, c);
    }
}

__global__ void __launch_bounds__(256) pair_coef_kernel(const int32_t *__restrict__ pair_i,
                                                        const int32_t *__restrict__ pair_j,
                                                        const float *__restrict__ pair_p, int64_t E, int K,
                                                        uint64_t seed, const float *__restrict__ adv,
                                                        const float *__restrict__ sumA, float *__restrict__ ce) {
    float SA = *sumA;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
        int i = pair_i[e], j = pair_j[e];
        float p = pair_p[e];
        float s = 0.f, c = 0.f;
        for (int g = 0; 4 * g < K; ++g) {
            uint4 u4 = edge_words(seed, i, j, g);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                int k = 4 * g + w;
                if (k < K && word_uniform(pick(u4, w)) < p) {
                    float y = __fsub_rn(adv[k], c), t = __fadd_rn(s, y);
                    c = __fsub_rn(__fsub_rn(t, s), y);
                    s = t;
                }
            }
        }
        float sum = __fsub_rn(s, c);
        ce[e] = __fdiv_rn(__fsub_rn(sum, __fmul_rn(p, SA)), float(K));
    }
}

__global__ void __launch_bounds__(256) endpoint_count_kernel(const int32_t *__restrict__ pair_i,
                                                             const int32_t *__restrict__ pair_j, int64_t E,
                                                             uint32_t *fcnt, uint32_t *rcnt) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
        atomicAdd(&fcnt[pair_i[e]], 1u);
        atomicAdd(&rcnt[pair_j[e]], 1u);
    }
}

__global__ void __launch_bounds__(256) reverse_fill_kernel(const int32_t *__restrict__ pair_j, int64_t E,
                                                           uint32_t *cursor, int32_t *__restrict__ rev) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x)
        rev[atomicAdd(&cursor[pair_j[e]], 1u)] = int32_t(e);
}

__device__ __forceinline__ void kacc(float &s, float &c, float x) {
    float y = __fsub_rn(x, c), t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__global__ void __launch_bounds__(256) grad_gather_kernel(const float *__restrict__ pos, int64_t N, float L, bool wrap,
                                                          const int32_t *__restrict__ pair_i,
                                                          const int32_t *__restrict__ pair_j,
                                                          const float *__restrict__ pair_d,
                                                          const float *__restrict__ ce,
                                                          const uint32_t *__restrict__ foff,
                                                          const uint32_t *__restrict__ roff,
                                                          const int32_t *__restrict__ rev, int form, float coef,
                                                          float *__restrict__ g_pos) {
    float hL = 0.5f * L;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        float xi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xi[a] = pos[3 * i + a];
            if (wrap) xi[a] = wrap_coord(xi[a], L);
        }
        float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
        for (int pass = 0; pass < 2; ++pass) {
            uint32_t e0 = pass == 0 ? foff[i] : roff[i], e1 = pass == 0 ? foff[i + 1] : roff[i + 1];
            for (uint32_t t = e0; t < e1; ++t) {
                int64_t e = pass == 0 ? int64_t(t) : int64_t(rev[t]);
                int other = pass == 0 ? pair_j[e] : pair_i[e];
                float d = pair_d[e];
                float fac = form == 0 ? (d > 0.f ? __fdiv_rn(coef, d) : 0.f) : __fmul_rn(2.0f, coef);
                float w = __fmul_rn(ce[e], fac);
                if (pass == 1) w = -w;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float xo = pos[3 * int64_t(other) + a];
                    if (wrap) xo = wrap_coord(xo, L);
                    // (x_j - x_i)_mi with i the pair's first index
                    float dx = pass == 0 ? min_image(xo, xi[a], L, hL) : min_image(xi[a], xo, L, hL);
                    kacc(s[a], c[a], __fmul_rn(w, dx));
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) g_pos[3 * i + a] = __fsub_rn(s[a], c[a]);
    }
}

size_t grad_layout(int64_t N, int64_t E, GradBuffers *gb, void *base) {
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    GradBuffers g;
    int64_t Ee = E > 0 ? E : 1;
    g.ce = reinterpret_cast<float *>(take(sizeof(float) * size_t(Ee)));
    g.fcnt = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N + 1)));
    g.foff = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N + 1)));
    g.rcnt = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N + 1)));
    g.roff = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N + 1)));
    g.cursor = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N)));
    g.rev = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * size_t(Ee)));
    g.sumA = reinterpret_cast<float *>(take(sizeof(float)));
    g.scan_tmp = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * scan_tmp_words(N)));
    g.seglist_words = segsort_list_words(Ee > N ? Ee : N);
    g.seglist = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(g.seglist_words)));
    if (gb) *gb = g;
    return off;
}

void launch_reinforce_grad(const float *pos, int64_t N, float L, bool wrap, const int32_t *pair_i,
                           const int32_t *pair_j, const float *pair_d, const float *pair_p, int64_t E, int32_t K,
                           uint64_t seed, const float *adv, int form, float coef, const GradBuffers &gb,
                           float *g_pos, cudaStream_t s) {
    sum_adv_kernel<<<1, 32, 0, s>>>(adv, K, gb.sumA);
    cudaMemsetAsync(gb.fcnt, 0, sizeof(uint32_t) * size_t(N + 1), s);
    cudaMemsetAsync(gb.rcnt, 0, sizeof(uint32_t) * size_t(N + 1), s);
    if (E > 0) {
        {
            JFOF_TRACE("grad_coef", s);
            pair_coef_kernel<<<grid_for(E, 256), 256, 0, s>>>(pair_i, pair_j, pair_p, E, K, seed, adv, gb.sumA, gb.ce);
        }
        JFOF_TRACE("grad_adjacency", s);
        endpoint_count_kernel<<<grid_for(E, 256), 256, 0, s>>>(pair_i, pair_j, E, gb.fcnt, gb.rcnt);
    }
    scan_exclusive(LoadCnt{gb.fcnt}, N, gb.foff, gb.scan_tmp, s);
    scan_exclusive(LoadCnt{gb.rcnt}, N, gb.roff, gb.scan_tmp, s);
    if (E > 0) {
        cudaMemcpyAsync(gb.cursor, gb.roff, sizeof(uint32_t) * size_t(N), cudaMemcpyDeviceToDevice, s);
        reverse_fill_kernel<<<grid_for(E, 256), 256, 0, s>>>(pair_j, E, gb.cursor, gb.rev);
        launch_segsort(gb.roff, N, gb.rev, E, s, nullptr, gb.seglist, gb.seglist_words);
    }
    {
        JFOF_TRACE("grad_gather", s);
        grad_gather_kernel<<<grid_for(N, 256), 256, 0, s>>>(pos, N, L, wrap, pair_i, pair_j, pair_d, gb.ce, gb.foff,
                                                            gb.roff, gb.rev, form, coef, g_pos);
    }
}

// ---------------------------------------------------------------------------
__global__ void eval_exp_kernel(const float *x, float *y, int64_t n) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x)
        y[t] = jexp(x[t]);
}

__global__ void eval_uniform_kernel(uint64_t seed, const int32_t *i, const int32_t *j, const int32_t *k, float *u,
                                    int64_t n) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        uint4 w = edge_words(seed, i[t], j[t], k[t] >> 2);
        u[t] = word_uniform(pick(w, k[t] & 3));
    }
}

void launch_eval_exp(const float *x, float *y, int64_t n, cudaStream_t s) {
    eval_exp_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
}

void launch_eval_uniform(uint64_t seed, const int32_t *i, const int32_t *j, const int32_t *k, float *u, int64_t n,
                         cudaStream_t s) {
    eval_uniform_kernel<<<grid_for(n, 256), 256, 0, s>>>(seed, i, j, k, u, n);
}

}  // namespace jfof
