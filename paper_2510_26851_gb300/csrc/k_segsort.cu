// k_segsort.cu -- ascending sort of many int32 segments (one warp each):
// <= 32 elements in registers (bitonic over shuffles), <= kSegWarpSmem in
// shared memory, larger ones in place in global memory (slow path).  Used to
// give the REINFORCE pair list and its reverse adjacency a fixed order.
#include "jfof_internal.cuh"
#include "k_reinforce.cuh"

namespace jfof {

constexpr int kSegWarps = 4;
constexpr int kSegWarpSmem = 2048;

// Sorting network with ascending comparators only ("flip" then halving
// steps), so a segment of any length behaves as if padded with +inf.
template <class Acc>
__device__ void warp_sort_network(Acc a, int m, int lane) {
    int P = 1;
    while (P < m) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < P; t += 32) {
                int u = (j == (k >> 1)) ? (t ^ (k - 1)) : (t ^ j);
                if (u > t && u < m) {
                    int x = a.get(t), y = a.get(u);
                    if (x > y) {
                        a.set(t, y);
                        a.set(u, x);
                    }
                }
            }
            __syncwarp();
        }
    }
}

struct PtrAcc {
    int *p;
    __device__ __forceinline__ int get(int i) const { return p[i]; }
    __device__ __forceinline__ void set(int i, int v) const { p[i] = v; }
};

__global__ void __launch_bounds__(32 * kSegWarps) segsort_kernel(const uint32_t *__restrict__ off, int64_t S,
                                                                 const int32_t *__restrict__ S_dev, int64_t cap,
                                                                 int32_t *__restrict__ data) {
    if (S_dev && int64_t(*S_dev) < S) S = *S_dev;
    __shared__ int buf[kSegWarps][kSegWarpSmem];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t sgi = int64_t(blockIdx.x) * kSegWarps + w; sgi < S; sgi += int64_t(gridDim.x) * kSegWarps) {
        uint32_t s0 = off[sgi];
        int m = int(off[sgi + 1] - s0);
        if (m <= 1 || int64_t(off[sgi + 1]) > cap) continue;
        int32_t *d = data + s0;
        if (m <= 32) {
            int v = lane < m ? d[lane] : INT_MAX;
            for (int k = 2; k <= 32; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    int u = __shfl_xor_sync(0xffffffffu, v, j);
                    bool up = (lane & k) == 0, lower = (lane & j) == 0;
                    v = (lower == up) ? min(v, u) : max(v, u);
                }
            if (lane < m) d[lane] = v;
        } else if (m <= kSegWarpSmem) {
            int *b = buf[w];
            for (int t = lane; t < m; t += 32) b[t] = d[t];
            __syncwarp();
            warp_sort_network(PtrAcc{b}, m, lane);
            for (int t = lane; t < m; t += 32) d[t] = b[t];
            __syncwarp();
        } else {
            warp_sort_network(PtrAcc{d}, m, lane);
        }
    }
}

void launch_segsort(const uint32_t *off, int64_t S, int32_t *data, int64_t cap, cudaStream_t s,
                    const int32_t *S_dev) {
    JFOF_TRACE("segsort", s);
    segsort_kernel<<<grid_for(S * 32, 32 * kSegWarps, 8), 32 * kSegWarps, 0, s>>>(off, S, S_dev, cap, data);
}

}  // namespace jfof
