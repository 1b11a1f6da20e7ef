// k_segsort.cu -- ascending sort of many int32 segments.
//
// Every segment runs the same ascending-only bitonic network ("flip" step,
// then halving steps) on P = next power of two >= m elements, the positions
// past m behaving as +inf.  Where the network runs depends on m:
//   m <= 256           one warp, the segment in registers (R = P/32 values a
//                      lane, element t = r*32 + lane): steps whose partner is
//                      in another lane use shuffles, the others swap registers
//   256 < m <= 1024    listed by the warp kernel, then one warp per segment
//                      with the segment in registers again (16 or 32 values a
//                      lane), in a kernel of its own so the short segments keep
//                      the smaller register footprint
//   m  > 1024          listed too, then one block per segment: in shared
//                      memory when P <= kSegSmem, otherwise chunks of kSegSmem
//                      sorted in shared memory and the long steps in global
//                      memory
// A segment that finds the list full is sorted in place in global memory by
// its warp (slow, but any list capacity is correct).  Used for the members
// of each halo and for the REINFORCE pair list and its reverse adjacency.
#include "jfof_internal.cuh"
#include "k_reinforce.cuh"

namespace jfof {

constexpr int kSegWarps = 8;
constexpr int kSegRegMax = 256;
constexpr int kSegMidMax = 1024;
constexpr int kSegBlock = 256;
constexpr int kSegSmem = 8192;
constexpr int kSegLogSmem = 13;

// Register network over P = 2^LOGP elements (LOGP >= 5).
template <int LOGP>
__device__ __forceinline__ void reg_sort(int32_t *d, int m, int lane) {
    constexpr int R = (1 << LOGP) / 32;
    int v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = r * 32 + lane;
        v[r] = t < m ? d[t] : INT_MAX;
    }
#pragma unroll
    for (int lk = 1; lk <= LOGP; ++lk) {
#pragma unroll
        for (int lj = lk - 1; lj >= 0; --lj) {
            const int X = (lj == lk - 1) ? (1 << lk) - 1 : (1 << lj);  // partner = t ^ X
            const int hb = 1 << lj;                                    // top bit of X
            const int Xl = X & 31, Xr = X >> 5;
            if (Xr == 0) {
                const bool lower = (lane & hb) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int p = __shfl_xor_sync(0xffffffffu, v[r], Xl);
                    v[r] = lower ? min(v[r], p) : max(v[r], p);
                }
            } else if (Xl == 0) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int q = r ^ Xr;
                    if (q > r) {
                        int a = v[r], b = v[q];
                        v[r] = min(a, b);
                        v[q] = max(a, b);
                    }
                }
            } else {  // flip across registers and lanes: Xl == 31
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int q = r ^ Xr;
                    if (q > r) {
                        int pr = __shfl_xor_sync(0xffffffffu, v[q], 31);
                        int pq = __shfl_xor_sync(0xffffffffu, v[r], 31);
                        v[r] = min(v[r], pr);
                        v[q] = max(v[q], pq);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = r * 32 + lane;
        if (t < m) d[t] = v[r];
    }
}

// One compare-exchange step (partner t ^ X, X's top bit hb) over the pairs
// t < u < lim of a[0, P), spread over the threads [tid, tid + nthr).
__device__ __forceinline__ void cx_step(int32_t *a, int P, int lim, int X, int hb, int tid, int nthr) {
    for (int c = tid; c < (P >> 1); c += nthr) {
        int t = ((c & ~(hb - 1)) << 1) | (c & (hb - 1));
        int u = t ^ X;
        if (u < lim) {
            int x = a[t], y = a[u];
            if (x > y) {
                a[t] = y;
                a[u] = x;
            }
        }
    }
}

// Fallback for a segment that found the list full: its warp, in place.
__device__ void warp_sort_global(int32_t *d, int m, int lane) {
    int P = 1, lp = 0;
    while (P < m) P <<= 1, ++lp;
    for (int lk = 1; lk <= lp; ++lk)
        for (int lj = lk - 1; lj >= 0; --lj) {
            int X = (lj == lk - 1) ? (1 << lk) - 1 : (1 << lj);
            cx_step(d, P, m, X, 1 << lj, lane, 32);
            __syncwarp();
        }
}

__global__ void __launch_bounds__(32 * kSegWarps) segsort_warp_kernel(const uint32_t *__restrict__ off, int64_t S,
                                                                      const int32_t *__restrict__ S_dev, int64_t cap,
                                                                      int32_t *__restrict__ data,
                                                                      uint32_t *__restrict__ list, int64_t list_cap) {
    if (S_dev && int64_t(*S_dev) < S) S = *S_dev;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t sgi = w0; sgi < S; sgi += nw) {
        uint32_t s0 = off[sgi], s1 = off[sgi + 1];
        int64_t m = int64_t(s1) - int64_t(s0);
        if (m <= 1 || int64_t(s1) > cap) continue;
        int32_t *d = data + s0;
        int mm = int(m);
        if (mm > kSegRegMax) {
            uint32_t slot = 0;
            if (lane == 0) slot = atomicAdd(list, 1u);
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (int64_t(slot) < list_cap)
                list[1 + slot] = uint32_t(sgi);
            else
                warp_sort_global(d, mm, lane);
        } else if (mm <= 32) {
            reg_sort<5>(d, mm, lane);
        } else if (mm <= 64) {
            reg_sort<6>(d, mm, lane);
        } else if (mm <= 128) {
            reg_sort<7>(d, mm, lane);
        } else {
            reg_sort<8>(d, mm, lane);
        }
    }
}

// Full network on a shared-memory tile of 2^lp elements (padded with +inf).
__device__ void smem_network(int32_t *b, int lp, int lk_lo, int tid) {
    int P = 1 << lp;
    for (int lk = lk_lo; lk <= lp; ++lk)
        for (int lj = lk - 1; lj >= 0; --lj) {
            int X = (lj == lk - 1) ? (1 << lk) - 1 : (1 << lj);
            cx_step(b, P, P, X, 1 << lj, tid, kSegBlock);
            __syncthreads();
        }
}

__device__ void tile_load(int32_t *b, const int32_t *d, int64_t base, int64_t m, int P, int tid) {
    for (int i = tid; i < P; i += kSegBlock) b[i] = base + i < m ? d[base + i] : INT_MAX;
    __syncthreads();
}

__device__ void tile_store(const int32_t *b, int32_t *d, int64_t base, int64_t m, int P, int tid) {
    for (int i = tid; i < P; i += kSegBlock)
        if (base + i < m) d[base + i] = b[i];
    __syncthreads();
}

// Listed segments of at most kSegMidMax members: one warp each, in registers.
__global__ void __launch_bounds__(32 * kSegWarps) segsort_mid_kernel(const uint32_t *__restrict__ off,
                                                                     int32_t *__restrict__ data,
                                                                     const uint32_t *__restrict__ list,
                                                                     int64_t list_cap) {
    int64_t n = list[0];
    if (n > list_cap) n = list_cap;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t e = w0; e < n; e += nw) {
        const uint32_t sgi = list[1 + e];
        const uint32_t s0 = off[sgi];
        const int m = int(off[sgi + 1] - s0);
        if (m > kSegMidMax) continue;
        if (m <= 512)
            reg_sort<9>(data + s0, m, lane);
        else
            reg_sort<10>(data + s0, m, lane);
    }
}

__global__ void __launch_bounds__(kSegBlock) segsort_block_kernel(const uint32_t *__restrict__ off,
                                                                  int32_t *__restrict__ data,
                                                                  const uint32_t *__restrict__ list,
                                                                  int64_t list_cap) {
    __shared__ int32_t buf[kSegSmem];
    int64_t n = list[0];
    if (n > list_cap) n = list_cap;
    const int tid = threadIdx.x;
    for (int64_t e = blockIdx.x; e < n; e += gridDim.x) {
        uint32_t sgi = list[1 + e];
        uint32_t s0 = off[sgi];
        int64_t m = int64_t(off[sgi + 1]) - int64_t(s0);
        if (m <= kSegMidMax) continue;  // the register kernel's
        int32_t *d = data + s0;
        int lp = 0;
        while ((int64_t(1) << lp) < m) ++lp;
        if (lp <= kSegLogSmem) {
            tile_load(buf, d, 0, m, 1 << lp, tid);
            smem_network(buf, lp, 1, tid);
            tile_store(buf, d, 0, m, 1 << lp, tid);
            continue;
        }
        // sort every kSegSmem chunk (all steps with k <= kSegSmem stay inside one)
        for (int64_t c = 0; c < m; c += kSegSmem) {
            tile_load(buf, d, c, m, kSegSmem, tid);
            smem_network(buf, kSegLogSmem, 1, tid);
            tile_store(buf, d, c, m, kSegSmem, tid);
        }
        int64_t P = int64_t(1) << lp;
        for (int lk = kSegLogSmem + 1; lk <= lp; ++lk) {
            // long steps in global memory
            for (int lj = lk - 1; lj >= kSegLogSmem; --lj) {
                int64_t X = (lj == lk - 1) ? (int64_t(1) << lk) - 1 : (int64_t(1) << lj);
                int64_t hb = int64_t(1) << lj;
                for (int64_t cc = tid; cc < (P >> 1); cc += kSegBlock) {
                    int64_t t = ((cc & ~(hb - 1)) << 1) | (cc & (hb - 1));
                    int64_t u = t ^ X;
                    if (u < m) {
                        int x = d[t], y = d[u];
                        if (x > y) {
                            d[t] = y;
                            d[u] = x;
                        }
                    }
                }
                __syncthreads();
            }
            // the halving steps below kSegSmem inside each chunk
            for (int64_t c = 0; c < m; c += kSegSmem) {
                tile_load(buf, d, c, m, kSegSmem, tid);
                for (int lj = kSegLogSmem - 1; lj >= 0; --lj) {
                    cx_step(buf, kSegSmem, kSegSmem, 1 << lj, 1 << lj, tid, kSegBlock);
                    __syncthreads();
                }
                tile_store(buf, d, c, m, kSegSmem, tid);
            }
        }
    }
}

int64_t segsort_list_words(int64_t cap) { return cap / (kSegRegMax + 1) + 2; }

void launch_segsort(const uint32_t *off, int64_t S, int32_t *data, int64_t cap, cudaStream_t s, const int32_t *S_dev,
                    uint32_t *list, int64_t list_words) {
    JFOF_TRACE("segsort", s);
    int64_t list_cap = list_words - 1;
    cudaMemsetAsync(list, 0, sizeof(uint32_t), s);
    segsort_warp_kernel<<<grid_for(S * 8, 32 * kSegWarps, 8), 32 * kSegWarps, 0, s>>>(off, S, S_dev, cap, data,
                                                                                       list, list_cap);
    segsort_mid_kernel<<<grid_for(list_cap * 32, 32 * kSegWarps, 8), 32 * kSegWarps, 0, s>>>(off, data, list,
                                                                                            list_cap);
    segsort_block_kernel<<<grid_for(list_cap * kSegBlock, kSegBlock, 4), kSegBlock, 0, s>>>(off, data, list,
                                                                                           list_cap);
}

}  // namespace jfof
