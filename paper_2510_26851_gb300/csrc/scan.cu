// scan.cu -- host side of the device-wide exclusive scan (tile sums).
#include "jfof_internal.cuh"

namespace jfof {

// One block scans up to kScanTile tile sums in place; sums[nt] = total.
__global__ void scan_single_block_kernel(uint32_t *sums, int64_t nt) {
    __shared__ uint32_t warps[kScanThreads / 32];
    int64_t base = int64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < nt ? sums[i] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t pre = block_exclusive_scan(s, warps, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < nt) sums[i] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0) sums[nt] = total;
}

size_t scan_tmp_words(int64_t n) {
    size_t words = 0;
    int64_t m = n;
    do {
        int64_t nt = (m + kScanTile - 1) / kScanTile;
        if (nt < 1) nt = 1;
        words += size_t(nt) + 1;
        m = nt;
    } while (m > kScanTile);
    return words + 64;
}

void scan_tiles_inplace(uint32_t *sums, int64_t nt, uint32_t *tmp, cudaStream_t s) {
    if (nt <= kScanTile) {
        scan_single_block_kernel<<<1, kScanThreads, 0, s>>>(sums, nt);
        return;
    }
    scan_exclusive(LoadU32{sums}, nt, sums, tmp, s);
}

}  // namespace jfof
