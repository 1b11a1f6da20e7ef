// k_tail.cu -- a6/a7 from the slot-ordered union-find forest: raw labels
// (Sec. 2 step (v)), the minimum-size cut with halo ids ascending by raw
// label, counts and CSR members (step (vi); Algorithms 1-2 "Compaction").
//
// Everything that depends on the component is computed in slot order, where
// the members of one component sit close together (same or neighbouring
// cells), and only the final per-particle outputs go to original order:
//   roots    parent[s] <- root r; per root the smallest original index
//            (the raw label) and the size, warp-aggregated
//   flags    one bit per raw label of a kept group (size >= min_size)
//   codes    halo id of a kept root = rank of its raw label among the set
//            bits (popcount prefix), so ids ascend by raw label
//   part.    members appended per halo (warp-aggregated cursors); one
//            (orig, code) record per particle partitioned into buckets of
//            2^shift consecutive original indices
//   scatter  the records bucket after bucket into label[] and halo_id[]:
//            the writes in flight cover one bucket, which stays in L2.  A
//            particle alone in its component and not a halo (about 46% of
//            them in the clustered boxes) gets no record: label[] is first
//            filled with the own index and halo_id[] with -1
// The members of each halo are then sorted ascending (segmented sort).
#include "jfof_internal.cuh"
#include "k_fof.cuh"
#include "k_reinforce.cuh"

namespace jfof {

constexpr int kTailThreads = 256;
// Code of a root whose component is the particle alone (and not a halo): it
// gets no record; its label (its own index) and halo id (-1) are pre-filled.
constexpr int32_t kSingleton = -2;
constexpr int kTailItems = 16;
constexpr int kTailTile = kTailThreads * kTailItems;
constexpr int kTailBPT = kTailBuckets / kTailThreads;  // bucket counters per thread
static_assert(kTailBuckets % kTailThreads == 0, "bucket counters split evenly over the threads");

namespace {

struct TailView {
    int *rootmin;     // [N] smallest original index of the root's component
    uint32_t *rsize;  // [N] component size at the root; then its halo id, -1 or kSingleton
    uint2 *rec;       // [N] (orig, code) grouped by bucket of orig
};

TailView tail_view(const FofBuffers &fb, int64_t N) {
    uint32_t *w = reinterpret_cast<uint32_t *>(fb.tmp);
    return TailView{reinterpret_cast<int *>(w), w + N, reinterpret_cast<uint2 *>(w + 2 * N)};
}

int bucket_shift(int64_t N) {
    int s = 12;
    while (((N - 1) >> s) + 1 > kTailBuckets) ++s;
    return s;
}

}  // namespace

__global__ void __launch_bounds__(256) tail_roots_kernel(const float4 *__restrict__ spos, int64_t N, int *parent,
                                                         int *__restrict__ rootmin, uint32_t *__restrict__ rsize) {
    const int lane = threadIdx.x & 31;
    for (int64_t w0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x - lane; w0 < N;
         w0 += int64_t(gridDim.x) * blockDim.x) {
        int64_t s = w0 + lane;
        bool ok = s < N;
        int r = -1, orig = INT_MAX;
        if (ok) {
            r = uf_find_ro(parent, int(s));
            orig = __float_as_int(spos[s].w);
            parent[s] = r;
        }
        unsigned grp = __match_any_sync(0xffffffffu, r);
        int mn = __reduce_min_sync(grp, orig);
        if (ok && lane == __ffs(grp) - 1) {
            atomicMin(&rootmin[r], mn);
            atomicAdd(&rsize[r], uint32_t(__popc(grp)));
        }
    }
}

__global__ void __launch_bounds__(256) tail_flags_kernel(const int *__restrict__ parent, int64_t N,
                                                         const int *__restrict__ rootmin,
                                                         const uint32_t *__restrict__ rsize, uint32_t min_size,
                                                         uint32_t *__restrict__ bits) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        if (parent[s] != int(s) || rsize[s] < min_size) continue;
        int l = rootmin[s];
        atomicOr(&bits[l >> 5], 1u << (l & 31));
    }
}

struct PopcWord {
    const uint32_t *bits;
    __device__ __forceinline__ uint32_t operator()(int64_t w) const { return uint32_t(__popc(bits[w])); }
};

__global__ void __launch_bounds__(256) tail_codes_kernel(const int *__restrict__ parent, int64_t N,
                                                         const int *__restrict__ rootmin, uint32_t *rsize,
                                                         uint32_t min_size, const uint32_t *__restrict__ bits,
                                                         const uint32_t *__restrict__ prefix, int64_t W,
                                                         int32_t *__restrict__ count, int32_t *__restrict__ hlabel,
                                                         int32_t *__restrict__ n_halos) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < N; s += int64_t(gridDim.x) * blockDim.x) {
        if (parent[s] != int(s)) continue;
        uint32_t n = rsize[s];
        int32_t code = n == 1u ? kSingleton : -1;
        if (n >= min_size) {
            int l = rootmin[s];
            uint32_t h = prefix[l >> 5] + uint32_t(__popc(bits[l >> 5] & ((1u << (l & 31)) - 1u)));
            count[h] = int32_t(n);
            hlabel[h] = l;
            code = int32_t(h);
        }
        rsize[s] = uint32_t(code);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_halos = int32_t(prefix[W]);
}

// Per root, GROUPS reads its code (halo id, -1, or kSingleton) from code_of;
// the labels-only form reads its component size from size_of (1: singleton).
template <bool GROUPS>
__global__ void __launch_bounds__(kTailThreads) tail_partition_kernel(
    const float4 *__restrict__ spos, int64_t N, const int *__restrict__ parent, const int *__restrict__ rootmin,
    const int32_t *__restrict__ code_of, const uint32_t *__restrict__ size_of, uint32_t *__restrict__ cursor,
    int32_t *__restrict__ members,
    uint32_t *__restrict__ bucket_fill, int shift, uint2 *__restrict__ rec) {
    __shared__ uint32_t hist[kTailBuckets], lstart[kTailBuckets], gbase[kTailBuckets];
    __shared__ uint32_t warp_sums[kTailThreads / 32];
    __shared__ uint2 stage[kTailTile];
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t tile0 = int64_t(blockIdx.x) * kTailTile;
#pragma unroll
    for (int j = 0; j < kTailBPT; ++j) hist[tid * kTailBPT + j] = 0u;
    __syncthreads();
    uint32_t key[kTailItems], val[kTailItems], rank[kTailItems];
#pragma unroll
    for (int k = 0; k < kTailItems; ++k) {
        int64_t s = tile0 + int64_t(k) * kTailThreads + tid;
        bool ok = s < N;
        int orig = 0;
        int32_t code = -1;
        uint32_t y = 0u;
        bool single = false;
        if (ok) {
            int r = parent[s];
            orig = __float_as_int(spos[s].w);
            if (GROUPS) {
                code = code_of[r];
                single = code == kSingleton;
            } else {
                single = size_of[r] == 1u;
            }
            if (!single) y = code >= 0 ? (0x80000000u | uint32_t(code)) : uint32_t(rootmin[r]);
        }
        if (GROUPS) {
            // a warp's 32 consecutive slots: one cursor bump per halo present
            int32_t g = ok ? code : -1;
            unsigned grp = __match_any_sync(0xffffffffu, g);
            if (g >= 0) {
                int leader = __ffs(grp) - 1;
                uint32_t b = 0u;
                if (lane == leader) b = atomicAdd(&cursor[g], uint32_t(__popc(grp)));
                b = __shfl_sync(grp, b, leader);
                members[b + uint32_t(__popc(grp & ((1u << lane) - 1u)))] = orig;
            }
        }
        const bool rec_ok = ok && !single;  // a singleton's outputs are pre-filled
        key[k] = rec_ok ? uint32_t(orig) : 0xffffffffu;
        val[k] = y;
        rank[k] = rec_ok ? atomicAdd(&hist[uint32_t(orig) >> shift], 1u) : 0u;
    }
    __syncthreads();
    uint32_t c[kTailBPT], sum = 0u, total;
#pragma unroll
    for (int j = 0; j < kTailBPT; ++j) {
        c[j] = hist[tid * kTailBPT + j];
        sum += c[j];
    }
    uint32_t pre = block_exclusive_scan(sum, warp_sums, &total);
#pragma unroll
    for (int j = 0; j < kTailBPT; ++j) {
        const int b = tid * kTailBPT + j;
        lstart[b] = pre;
        gbase[b] = c[j] ? atomicAdd(&bucket_fill[b], c[j]) : 0u;
        pre += c[j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTailItems; ++k)
        if (key[k] != 0xffffffffu) stage[lstart[key[k] >> shift] + rank[k]] = make_uint2(key[k], val[k]);
    __syncthreads();
    // runs of one bucket go out contiguously
    for (uint32_t i = tid; i < total; i += kTailThreads) {
        uint2 e = stage[i];
        uint32_t b = e.x >> shift;
        rec[(int64_t(b) << shift) + gbase[b] + (i - lstart[b])] = e;
    }
}

// Records of bucket b sit at [b << shift, (b << shift) + fill[b]); labels and
// halo ids not written here were pre-filled (own index, -1).
template <bool GROUPS>
__global__ void __launch_bounds__(256) tail_scatter_kernel(const uint2 *__restrict__ rec, int64_t N,
                                                           const uint32_t *__restrict__ fill, int shift,
                                                           const int32_t *__restrict__ hlabel,
                                                           int32_t *__restrict__ label,
                                                           int32_t *__restrict__ halo_id) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= N) return;
    if (uint32_t(e - ((e >> shift) << shift)) >= fill[e >> shift]) return;
    uint2 r = rec[e];
    if (GROUPS && (r.y & 0x80000000u)) {
        int32_t h = int32_t(r.y & 0x7fffffffu);
        label[r.x] = hlabel[h];
        halo_id[r.x] = h;
    } else {
        label[r.x] = int32_t(r.y);
    }
}

__global__ void __launch_bounds__(256) iota_fill_kernel(int32_t *__restrict__ p, int64_t N) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = int32_t(i);
}

static void tail_roots(const FofBuffers &fb, const TailView &v, int64_t N, cudaStream_t s) {
    cudaMemsetAsync(v.rootmin, 0x7f, sizeof(int) * size_t(N), s);
    cudaMemsetAsync(v.rsize, 0, sizeof(uint32_t) * size_t(N), s);
    cudaMemsetAsync(fb.bucket_fill, 0, sizeof(uint32_t) * kTailBuckets, s);
    JFOF_TRACE("finalize_roots", s);
    tail_roots_kernel<<<grid_full(N, 256), 256, 0, s>>>(reinterpret_cast<const float4 *>(fb.spos), N, fb.parent,
                                                         v.rootmin, v.rsize);
}

void launch_tail_labels(const FofBuffers &fb, int64_t N, int32_t *label, cudaStream_t s) {
    TailView v = tail_view(fb, N);
    tail_roots(fb, v, N, s);
    int shift = bucket_shift(N);
    {
        JFOF_TRACE("finalize_labels", s);
        iota_fill_kernel<<<grid_for(N, 256), 256, 0, s>>>(label, N);
        tail_partition_kernel<false><<<unsigned((N + kTailTile - 1) / kTailTile), kTailThreads, 0, s>>>(
            fb.spos, N, fb.parent, v.rootmin, nullptr, v.rsize, nullptr, nullptr, fb.bucket_fill, shift, v.rec);
        tail_scatter_kernel<false><<<grid_full(N, 256), 256, 0, s>>>(v.rec, N, fb.bucket_fill, shift, nullptr, label,
                                                                      nullptr);
    }
}

void launch_tail_groups(const FofBuffers &fb, int64_t N, int32_t min_size, int64_t H_cap, const GroupBuffers &gb,
                        int32_t *label, int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members,
                        int32_t *n_halos, cudaStream_t s) {
    TailView v = tail_view(fb, N);
    tail_roots(fb, v, N, s);
    int64_t W = (N + 31) / 32;
    uint32_t *bits = gb.cnt, *prefix = gb.hid;
    cudaMemsetAsync(bits, 0, sizeof(uint32_t) * size_t(W), s);
    cudaMemsetAsync(count, 0, sizeof(int32_t) * size_t(H_cap), s);
    {
        JFOF_TRACE("group_count", s);
        tail_flags_kernel<<<grid_for(N, 256), 256, 0, s>>>(fb.parent, N, v.rootmin, v.rsize, uint32_t(min_size),
                                                           bits);
        scan_exclusive(PopcWord{bits}, W, prefix, gb.scan_tmp, s);
        tail_codes_kernel<<<grid_for(N, 256), 256, 0, s>>>(fb.parent, N, v.rootmin, v.rsize, uint32_t(min_size),
                                                           bits, prefix, W, count, gb.hlabel, n_halos);
    }
    {
        JFOF_TRACE("scan", s);
        scan_exclusive(LoadU32{reinterpret_cast<const uint32_t *>(count)}, H_cap,
                       reinterpret_cast<uint32_t *>(halo_start), gb.scan_tmp, s);
    }
    cudaMemcpyAsync(gb.cursor, halo_start, sizeof(uint32_t) * size_t(H_cap), cudaMemcpyDeviceToDevice, s);
    int shift = bucket_shift(N);
    {
        JFOF_TRACE("members_fill", s);
        tail_partition_kernel<true><<<unsigned((N + kTailTile - 1) / kTailTile), kTailThreads, 0, s>>>(
            fb.spos, N, fb.parent, v.rootmin, reinterpret_cast<const int32_t *>(v.rsize), nullptr, gb.cursor,
            members, fb.bucket_fill, shift, v.rec);
    }
    {
        JFOF_TRACE("finalize_labels", s);
        iota_fill_kernel<<<grid_for(N, 256), 256, 0, s>>>(label, N);
        cudaMemsetAsync(halo_id, 0xff, sizeof(int32_t) * size_t(N), s);
        tail_scatter_kernel<true><<<grid_full(N, 256), 256, 0, s>>>(v.rec, N, fb.bucket_fill, shift, gb.hlabel, label,
                                                                     halo_id);
    }
    launch_segsort(reinterpret_cast<const uint32_t *>(halo_start), H_cap, members, N, s, n_halos, gb.seglist,
                   gb.seglist_words);
}

}  // namespace jfof
