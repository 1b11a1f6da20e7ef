// k_groups.cu -- a7: compaction, histogram, minimum-size cut and CSR members
// (Sec. 2 step (vi); Algorithms 1-2 "Compaction").
//
//   cnt[r]      members of the component whose raw label is r
//   hid         exclusive scan of [label[r] == r && cnt[r] >= min_size]
//               -> halo ids ascending by raw label, H = hid[N]
//   halo_id[i]  hid[label[i]] when the group survives the cut, else -1
//   halo_start  exclusive scan of count[0..H_cap)
//   members     original indices grouped by halo, sorted ascending in each
//               halo so that every later reduction runs in a fixed order
#include "jfof_internal.cuh"
#include "k_fof.cuh"
#include "k_reinforce.cuh"

namespace jfof {

__global__ void __launch_bounds__(256) group_count_kernel(const int32_t *__restrict__ label, int64_t N,
                                                          uint32_t *__restrict__ cnt, DevStatus st) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        int32_t l = label[i];
        if (l < 0 || int64_t(l) >= N) {
            latch(st, JFOF_EINVAL);
            continue;
        }
        atomicAdd(&cnt[l], 1u);
    }
}

struct RootFlag {
    const int32_t *label;
    const uint32_t *cnt;
    uint32_t min_size;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const {
        return (int64_t(label[i]) == i && cnt[i] >= min_size) ? 1u : 0u;
    }
};

__global__ void __launch_bounds__(256) group_assign_kernel(const int32_t *__restrict__ label, int64_t N,
                                                           const uint32_t *__restrict__ cnt,
                                                           const uint32_t *__restrict__ hid,
                                                           int32_t *__restrict__ halo_id, int32_t *__restrict__ count,
                                                           int32_t *__restrict__ n_halos) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        int32_t l = label[i];
        if (l < 0 || int64_t(l) >= N) {
            halo_id[i] = -1;
            continue;
        }
        uint32_t h = hid[l];
        bool kept = hid[l + 1] != h;
        halo_id[i] = kept ? int32_t(h) : -1;
        if (kept && int64_t(l) == i) count[h] = int32_t(cnt[l]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_halos = int32_t(hid[N]);
}

struct LoadCount {
    const int32_t *count;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return uint32_t(count[i]); }
};

__global__ void __launch_bounds__(256) members_fill_kernel(const int32_t *__restrict__ halo_id, int64_t N,
                                                           uint32_t *__restrict__ cursor,
                                                           int32_t *__restrict__ members) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        int32_t h = halo_id[i];
        if (h >= 0) members[atomicAdd(&cursor[h], 1u)] = int32_t(i);
    }
}

size_t groups_layout(int64_t N, int64_t H_cap, GroupBuffers *gb, void *base) {
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    GroupBuffers g;
    g.cnt = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N)));
    g.hid = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(N + 1)));
    g.cursor = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(H_cap + 1)));
    int64_t big = N > H_cap ? N : H_cap;
    g.scan_tmp = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * scan_tmp_words(big)));
    g.seglist_words = segsort_list_words(N);
    g.seglist = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * size_t(g.seglist_words)));
    g.hlabel = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * size_t(H_cap)));
    if (gb) *gb = g;
    return off;
}

void launch_groups(const int32_t *label, int64_t N, int32_t min_size, int64_t H_cap, const GroupBuffers &gb,
                   int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members, int32_t *n_halos,
                   const DevStatus &st, cudaStream_t s) {
    cudaMemsetAsync(gb.cnt, 0, sizeof(uint32_t) * size_t(N), s);
    cudaMemsetAsync(count, 0, sizeof(int32_t) * size_t(H_cap), s);
    {
        JFOF_TRACE("group_count", s);
        group_count_kernel<<<grid_for(N, 256), 256, 0, s>>>(label, N, gb.cnt, st);
    }
    { JFOF_TRACE("scan", s); scan_exclusive(RootFlag{label, gb.cnt, uint32_t(min_size)}, N, gb.hid, gb.scan_tmp, s); }
    {
        JFOF_TRACE("group_assign", s);
        group_assign_kernel<<<grid_for(N, 256), 256, 0, s>>>(label, N, gb.cnt, gb.hid, halo_id, count, n_halos);
    }
    { JFOF_TRACE("scan", s); scan_exclusive(LoadCount{count}, H_cap, reinterpret_cast<uint32_t *>(halo_start), gb.scan_tmp, s); }
    cudaMemcpyAsync(gb.cursor, halo_start, sizeof(uint32_t) * size_t(H_cap), cudaMemcpyDeviceToDevice, s);
    {
        JFOF_TRACE("members_fill", s);
        members_fill_kernel<<<grid_for(N, 256), 256, 0, s>>>(halo_id, N, gb.cursor, members);
    }
    // members of each halo ascending by original index (segments past H are empty)
    launch_segsort(reinterpret_cast<const uint32_t *>(halo_start), H_cap, members, N, s, n_halos, gb.seglist,
                   gb.seglist_words);
}

}  // namespace jfof
