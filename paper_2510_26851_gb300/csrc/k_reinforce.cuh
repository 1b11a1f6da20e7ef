// k_reinforce.cuh -- internal launchers of the REINFORCE topological mode.
#pragma once
#include "jfof_internal.cuh"

namespace jfof {

// Sorts data[off[t] .. off[t+1]) ascending for every t < S whose segment ends
// within cap elements (segments past cap are left alone).
// S_dev (may be null, device): a tighter segment count read by the kernel.
// list: device scratch of list_words uint32 for the segments longer than
// 1024; segsort_list_words(cap) words hold all of them, fewer only slow the
// overflow down.
int64_t segsort_list_words(int64_t cap);
void launch_segsort(const uint32_t *off, int64_t S, int32_t *data, int64_t cap, cudaStream_t s, const int32_t *S_dev,
                    uint32_t *list, int64_t list_words);

// Views into the pair-list workspace.
struct PairBuffers {
    uint32_t *cnt;   // [N] partners j > i per i
    uint32_t *off;   // [N+1] exclusive scan of cnt
    uint32_t *scan_tmp;
    unsigned long long *total;  // [1] 64-bit pair count
    uint32_t *seglist;          // segmented-sort list (bounded: overflow sorts in place)
    int64_t seglist_words;
    void *cells_ws;  // binning workspace (fof_layout at the pair-cut grid)
};
size_t pairs_layout(int64_t N, int n, PairBuffers *pb, void *base);

struct PairGeom {
    float L, hL, rc2, b, b2, coef, inv_cell;
    int n, nb, form;
    bool wrap;
};

void launch_pairs(const float *pos, int64_t N, const PairGeom &pg, const PairBuffers &pb, int64_t cap,
                  int32_t *pair_i, int32_t *pair_j, float *pair_d, float *pair_p, int64_t *n_pairs,
                  const DevStatus &st, cudaStream_t s);

// Sampling workspace: a chunk of per-sample size counters.
constexpr int kSampleChunk = 16;
size_t sample_layout(int64_t N, uint32_t **counts, void *base);
void launch_reinforce_sample(int64_t N, const int32_t *pair_i, const int32_t *pair_j, const float *pair_p, int64_t E,
                             int32_t K, uint64_t seed, int32_t min_size, uint32_t *counts, int32_t *labels,
                             int32_t *n_halos, const DevStatus &st, cudaStream_t s);

struct GradBuffers {
    float *ce;         // [E] per-pair coefficient
    uint32_t *fcnt;    // [N+1]
    uint32_t *foff;    // [N+1]
    uint32_t *rcnt;    // [N+1]
    uint32_t *roff;    // [N+1]
    uint32_t *cursor;  // [N]
    int32_t *rev;      // [E]
    float *sumA;       // [1]
    uint32_t *scan_tmp;
    uint32_t *seglist;  // segmented-sort list (bounded: overflow sorts in place)
    int64_t seglist_words;
};
size_t grad_layout(int64_t N, int64_t E, GradBuffers *gb, void *base);
void launch_reinforce_grad(const float *pos, int64_t N, float L, bool wrap, const int32_t *pair_i,
                           const int32_t *pair_j, const float *pair_d, const float *pair_p, int64_t E, int32_t K,
                           uint64_t seed, const float *adv, int form, float coef, const GradBuffers &gb,
                           float *g_pos, cudaStream_t s);

// Verification hooks: the device exponential and edge uniforms.
void launch_eval_exp(const float *x, float *y, int64_t n, cudaStream_t s);
void launch_eval_uniform(uint64_t seed, const int32_t *i, const int32_t *j, const int32_t *k, float *u, int64_t n,
                         cudaStream_t s);

}  // namespace jfof
