/*
 * jfof.h -- C ABI of the GB300 (sm_103a) Friends-of-Friends hot path.
 *
 * The operations follow Horowitz & Bayer, "jFoF: GPU Cluster Finding with
 * Gradient Propagation" (arXiv 2510.26851):
 *   - input normalisation and labels (Sec. 2 steps (i), (v)),
 *   - linked-cell candidate search over a periodic box (Sec. 2.2, Algorithm 2),
 *   - the linking criterion d <= b on minimum-image separations (Sec. 2 step
 *     (iv); Algorithm 2),
 *   - connected components as labels = smallest member index (the fixed point
 *     of the min-label propagation of Sec. 2 step (v) / Algorithm 2),
 *   - compaction to halo ids and per-halo counts (Sec. 2 step (vi)),
 *   - halo properties and their frozen-assignment adjoint (Sec. 3.1, Eq. 4,
 *     Table 1),
 *   - the REINFORCE topological mode (Sec. 3.2, Eqs. 6-8).
 *
 * Conventions shared by every call:
 *   - Every array argument is a DEVICE pointer owned by the caller, unless the
 *     argument's comment says "host".  The library never frees caller memory.
 *   - Scratch memory is passed in by the caller as (ws, ws_bytes); the matching
 *     *_bytes query gives the size.  No call allocates device memory except
 *     jfof_create (a few bytes of status words per context) and the CUDA
 *     graphs and streams that jfof_fof_batched and jfof_reinforce_sample
 *     create on first use and keep in the context.
 *   - Work is enqueued on the context's CUDA stream and the call returns without
 *     waiting, except where a comment says the call synchronises.
 *   - Particle indices are int32: N <= 2^31 - 1.  Positions are float32 AoS
 *     [N,3] in [0, L) unless JFOF_WRAP is given.
 *   - Return value: JFOF_OK or an error code.  Argument errors are detected on
 *     the host and nothing is enqueued.  Errors found by a kernel (a position
 *     outside the box, a bounded wait that ran out, an overflowed capacity) are
 *     latched in the context's device status word and returned by the next
 *     jfof_sync() (which also clears it).  A kernel that latches an error still
 *     keeps every memory access in bounds; its outputs are then unspecified.
 */
#ifndef JFOF_H
#define JFOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define JFOF_OK 0
#define JFOF_EINVAL 1    /* bad argument (null pointer, N < 1, b <= 0, b >= L/2, ...) */
#define JFOF_ERANGE 2    /* a position outside [0, L) without JFOF_WRAP, or not finite */
#define JFOF_ENOMEM 3    /* workspace smaller than the *_bytes query */
#define JFOF_ECUDA 4     /* a CUDA runtime call failed */
#define JFOF_ETIMEOUT 5  /* a bounded device loop ran out of iterations */
#define JFOF_EOVERFLOW 6 /* an output capacity was too small */

/* Flags. */
#define JFOF_WRAP 1u /* wrap positions into [0, L): x - L*floor(x/L), then >= L or < 0 -> 0
                        (Algorithm 2 "X mod L") */

typedef struct jfof_ctx jfof_ctx;

/* Create a context on CUDA device `device` that enqueues on `stream` (a
   cudaStream_t; NULL = the legacy default stream).  Allocates the context's
   device status word.  *ctx receives the handle. */
int jfof_create(jfof_ctx **ctx, int device, void *stream);

/* Destroy a context (synchronises its stream first). */
int jfof_destroy(jfof_ctx *ctx);

/* Change the stream later calls enqueue on. */
int jfof_set_stream(jfof_ctx *ctx, void *stream);

/* Synchronise the context's stream, then return and clear the latched device
   status (JFOF_OK if no kernel reported an error). */
int jfof_sync(jfof_ctx *ctx);

/* Static description of a status code. */
const char *jfof_strerror(int code);

/* Test hook for the bounded device loops: maximum iterations of every
   union-find retry loop (default 1<<24; 0 restores the default).  A loop that
   runs out latches JFOF_ETIMEOUT and returns. */
int jfof_set_loop_budget(jfof_ctx *ctx, int64_t iterations);

/* Per-launch tracing: with tracing on, every kernel the library launches is
   bracketed by CUDA events recorded on the context's stream.  jfof_trace_read
   synchronises the stream and writes one text line per kernel name,
   "name launches total_ms", into buf (at most len bytes, NUL-terminated), then
   forgets the records.  Returns JFOF_EOVERFLOW if buf is too small. */
int jfof_trace_enable(jfof_ctx *ctx, int on);
int jfof_trace_read(jfof_ctx *ctx, char *buf, size_t len, size_t *written);

/* Cell classes of the link step (see jfof_link): a cell with at most
   `small_max` particles (at most 255 is used) is "small" (its particles'
   candidate pairs are spread over a warp); one with more
   than `dense_over` (and at most 65535) is "dense" (linked through its
   sub-cells; 0 disables that path; -1, the default, takes 160 for boxes of
   more than 2^23 particles and 96 below); the rest are "medium" (one warp per
   cell).  Default small_max 16.  Labels do not depend on them; only speed does.
   Takes effect at the next jfof_bin_cells. */
int jfof_set_cell_classes(jfof_ctx *ctx, int32_t small_max, int32_t dense_over);

/* Tuning knob: warps per CTA of the four list-driven link kernels (medium
   cells local and cross, dense cells local and neighbours).  Shape 0 (the
   default) = (4, 8, 4, 8), 1 = all 8, 2 = all 4.  Labels do not depend on it. */
int jfof_set_cta_shape(jfof_ctx *ctx, int32_t shape);

/* ---------------------------------------------------------------------- */
/* Grid choice (Sec. 2.2, Algorithm 2 "Grid setup").                        */
/* The linked-cell grid has n cells per axis with cell side L/n >= 1.01 b,  */
/* so every pair within b lies in the same or adjacent cells (the printed   */
/* n = ceil(L/b) gives cells smaller than b; see the design notes).  n is 1 */
/* or >= 3.  Labels do not depend on n; it only changes speed.             */

/* Largest legal n for (L, b), capped at 1600. */
int jfof_max_cells_per_axis(float L, float b, int32_t *n_axis);

/* Default n for N particles: the largest legal n with n^3 <= N (at least 1),
   raised by up to max(2, n/8) when that is the smallest n at which the cells
   are narrow enough for the sub-cell path of dense cells (at most 9
   sub-cells of side <= b/(1.02 sqrt 3) per cell side). */
int jfof_default_cells_per_axis(int64_t N, float L, float b, int32_t *n_axis);

/* ---------------------------------------------------------------------- */
/* Plain FoF pipeline.                                                      */

/* Cell structure produced by jfof_bin_cells.  Its pointers point into the
   caller's workspace; the struct itself is plain data the caller keeps. */
typedef struct {
    int64_t n;            /* particles */
    int32_t n_axis;       /* cells per axis */
    int32_t brick;        /* cells per brick side (cell table is brick-major) */
    float L, b;           /* box side and linking length */
    uint32_t flags;       /* flags given to jfof_bin_cells */
    int32_t small_threshold; /* cells with at most this many particles are "small" */
    int32_t dense_threshold; /* cells with more particles take the dense path (0 = off) */
    void *spos;           /* device float4[n]: positions in cell order; .w holds the
                             bits of the int32 original index */
    uint32_t *cell_start; /* device [n_cells_table + 1]: start of each cell in spos */
    int64_t n_cells_table;/* entries of the brick-major cell table */
    void *workspace;      /* the workspace given to jfof_bin_cells; jfof_link uses
                             the rest of it (union-find forest, dense-cell tables) */
} jfof_cells;

/* Bytes of workspace for jfof_bin_cells + jfof_link with N particles and
   n_axis cells per axis. */
int jfof_fof_bytes(int64_t N, int32_t n_axis, size_t *bytes);

/* a1-a3: optional wrap, cell binning (cell key ix + n(iy + n iz) grouped into
   bricks of 16^3 cells), and a two-level counting sort of the particles by
   cell.  pos: device float32 [N,3].  Fills *cells (views into ws).
   Sec. 2 step (i); Algorithm 2 "Wrap positions", "Cell indexing",
   "Sort by cell".  Latches JFOF_ERANGE for a position outside [0, L)
   without JFOF_WRAP. */
int jfof_bin_cells(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b,
                   int32_t n_axis, uint32_t flags, void *ws, size_t ws_bytes,
                   jfof_cells *cells);

/* a4-a6: 27-cell neighbour scan (each unordered cell pair once), link test
   d2 <= b*b with d2 = (dx*dx + dy*dy) + dz*dz in binary32 without FMA on
   minimum-image differences, lock-free union-find, and the raw label
   label[i] = smallest original index in i's component, in original order.
   Dense cells are split into sub-cells of side <= b/(1.02 sqrt 3): pairs in
   one sub-cell are friends by geometry and are united without a test, and a
   sub-cell pair is tested only until its first link (the components are
   those of testing every pair).  label: device int32 [N].  Sec. 2 steps
   (iii)-(v); Sec. 2.2; Algorithm 2. */
int jfof_link(jfof_ctx *ctx, const jfof_cells *cells, int32_t *label);

/* Bytes of workspace for jfof_groups with N particles. */
int jfof_groups_bytes(int64_t N, size_t *bytes);

/* a7: compaction, histogram and minimum-size cut (Sec. 2 step (vi)).
   label: device int32 [N] raw labels (smallest member index).
   Outputs (device):
     halo_id   [N]       halo of each particle, ascending by raw label, -1 if
                         its group has fewer than min_size members;
     count     [H_cap]   members per halo;
     halo_start[H_cap+1] CSR offsets of members;
     members   [N]       original indices grouped by halo, ascending within a
                         halo (only the first halo_start[H] entries are used);
     n_halos   [1]       H.
   H_cap = N / min_size (the most halos that can exist). */
int jfof_groups(jfof_ctx *ctx, const int32_t *label, int64_t N, int32_t min_size,
                void *ws, size_t ws_bytes, int32_t *halo_id, int32_t *count,
                int32_t *halo_start, int32_t *members, int32_t *n_halos);

/* a8: halo properties (Sec. 3.1, Eq. 4; Table 1), binary32 with compensated
   sums in a fixed order (deterministic):
     mass[h]  = particle_mass * n_h
     com[h]   = wrap(x_r + (1/n_h) sum_i mi(x_i - x_r)), r = smallest member
     vmean[h] = (1/n_h) sum_i v_i
     sigv[h]  = sqrt((1/(3 n_h)) sum_i |v_i - vmean_h|^2)
   pos, vel: device float32 [N,3] (vel may be NULL: vmean and sigv untouched);
   positions are wrapped as in jfof_bin_cells when flags has JFOF_WRAP.
   halo_start, members, n_halos: from jfof_groups.  Outputs [H_cap] / [H_cap,3];
   entries h >= H are left untouched. */
int jfof_halo_props(jfof_ctx *ctx, const float *pos, const float *vel, int64_t N,
                    float L, uint32_t flags, const int32_t *halo_start,
                    const int32_t *members, const int32_t *n_halos, int64_t H_cap,
                    float particle_mass, float *mass, float *com, float *vmean,
                    float *sigv);

/* a9: frozen-assignment adjoint (Sec. 3.1, Eq. 4): with memberships fixed,
     g_pos_i = g_com[h] / n_h
     g_vel_i = g_vmean[h] / n_h + g_sigv[h] (v_i - vmean_h) / (3 n_h sigv_h)
   (the sigma term is 0 when sigv_h = 0); 0 for particles with halo_id -1.
   Any of g_com [H,3], g_vmean [H,3], g_sigv [H] may be NULL (zero).  vel,
   vmean and sigv may be NULL only when g_sigv is NULL.  Outputs g_pos,
   g_vel: device float32 [N,3] (either may be NULL to skip it). */
int jfof_halo_props_backward(jfof_ctx *ctx, const float *vel, const int32_t *halo_id,
                             const int32_t *count, int64_t N, const float *vmean,
                             const float *sigv, const float *g_com,
                             const float *g_vmean, const float *g_sigv, float *g_pos,
                             float *g_vel);

/* ---------------------------------------------------------------------- */
/* REINFORCE topological mode (Sec. 3.2, Eqs. 6-8).                        */

/* Host helper for the edge-probability constant `coef`:
     prob_form 0: p = sigmoid((b - d) / tau), coef = 1/tau (tau <= 0 means
                  tau = 0.05 b), computed in double and rounded once;
     prob_form 1: p = sigmoid(alpha (b^2 - d^2) / b^2) (Eq. 8),
                  coef = alpha / f32(b*b), computed in double, rounded once. */
int jfof_prob_coef(float b, int32_t prob_form, float tau, float alpha, float *coef);

/* a11: the fixed candidate list ("we do not rebuild the neighbor list",
   Sec. 3.2): every unordered pair i < j with d2 < r_cut*r_cut (d2 as in
   jfof_link), sorted by (i, j), with d = sqrt(d2) (IEEE) and the edge
   probability p = 1 / (1 + E(-z)), z = (b - d)*coef (form 0) or
   (b*b - d2)*coef (form 1); E is the library's binary32 exponential
   (Cody-Waite reduction + degree-7 Taylor, see jfof_eval_exp).
   Writes min(E, cap) pairs into pair_i/pair_j (int32) and pair_d/pair_p
   (float32), and the total E into *n_pairs (device int64).  cap = 0 only
   counts (the output pointers may then be NULL); E > cap > 0 latches
   JFOF_EOVERFLOW and writes no pairs.  E must fit in uint32. */
int jfof_pairs_bytes(int64_t N, float L, float r_cut, size_t *bytes);
int jfof_pairs(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, float r_cut,
               int32_t prob_form, float coef, uint32_t flags, void *ws, size_t ws_bytes,
               int64_t cap, int32_t *pair_i, int32_t *pair_j, float *pair_d, float *pair_p,
               int64_t *n_pairs);

/* a12: K stochastic topologies in one call (Eq. 8 Bernoulli edges over the
   fixed list).  Edge e is present in sample k iff u < p_e, where
   u = (w >> 8) * 2^-24 and w is word (k mod 4) of Philox4x32-10 (Salmon et
   al., SC'11) with key (seed low 32 bits, seed high 32 bits) and counter
   (min(i,j), max(i,j), floor(k/4), 0).  Outputs: labels [K, N] device int32,
   row k = smallest member index of each particle's component in sample k;
   n_halos [K] device int32 = components with >= min_size members.  E is the
   host pair count.  The pair arrays are from jfof_pairs.  All K samples run
   as ONE CUDA graph launch on the context's stream (chunks of 16 samples,
   so a chunk's label rows stay in L2); the graph is kept in the context and
   updated in place by later calls of the same shape. */
int jfof_reinforce_sample_bytes(int64_t N, size_t *bytes);
int jfof_reinforce_sample(jfof_ctx *ctx, int64_t N, const int32_t *pair_i, const int32_t *pair_j,
                          const float *pair_p, int64_t E, int32_t K, uint64_t seed,
                          int32_t min_size, void *ws, size_t ws_bytes, int32_t *labels,
                          int32_t *n_halos);

/* a13: score-function gradient with respect to positions (Eqs. 6-7):
     g = (1/K) sum_k A_k d log p(y_k) / dx,  d log p / dz_e = y_e - p_e,
   with y_ke regenerated from the same counter-based draws (no edge storage),
   advantage A [K] device float32 (e.g. L_k - mean L, the batch-mean baseline
   of Sec. 3.2), dz/dx_i = (x_j - x_i)_mi / (tau d) (form 0) or
   2 (alpha/b^2) (x_j - x_i)_mi (form 1), dz/dx_j = -dz/dx_i, and 0 for d = 0.
   Binary32 with compensated sums in a fixed order (deterministic).  The pairs
   must be sorted by i (as jfof_pairs writes them).  g_pos: device [N,3]. */
int jfof_reinforce_grad_bytes(int64_t N, int64_t E, size_t *bytes);
int jfof_reinforce_grad(jfof_ctx *ctx, const float *pos, int64_t N, float L, uint32_t flags,
                        const int32_t *pair_i, const int32_t *pair_j, const float *pair_d,
                        const float *pair_p, int64_t E, int32_t K, uint64_t seed,
                        const float *advantage, int32_t prob_form, float coef, void *ws,
                        size_t ws_bytes, float *g_pos);

/* Verification hooks: the device exponential E(x) used for edge
   probabilities, y[t] = E(x[t]); and the edge uniforms of jfof_reinforce_sample,
   u[t] for edge (i[t], j[t]) in sample k[t].  All arrays on the device. */
int jfof_eval_exp(jfof_ctx *ctx, const float *x, float *y, int64_t n);
int jfof_eval_edge_uniform(jfof_ctx *ctx, uint64_t seed, const int32_t *i, const int32_t *j,
                           const int32_t *k, float *u, int64_t n);

/* ---------------------------------------------------------------------- */
/* Batched FoF: many independent boxes (no counterpart in the paper; its   */
/* AI-systems form of Sec. 1's GPU-resident analysis).                     */

/* Bytes of workspace for jfof_fof_batched.  h_box_offset: host [B+1], box k
   holds particles [h_box_offset[k], h_box_offset[k+1]) of the concatenated
   arrays (h_box_offset[0] = 0, total <= 2^31-1); h_L, h_b: host [B];
   h_n_axis: host [B] cells per axis (0 or NULL = default). */
int jfof_batch_bytes(const int64_t *h_box_offset, int32_t B, const float *h_L, const float *h_b,
                     const int32_t *h_n_axis, int32_t min_size, size_t *bytes);

/* a1-a7 for B boxes: labels (smallest member index, numbered inside each
   box), halo ids (numbered from 0 inside each box, -1 below min_size) and
   n_halos [B], all device arrays over the concatenated particles.  Boxes
   never interact.  h_small / h_dense: host [B] per-box cell classes, h_shape:
   host [B] per-box CTA shapes of the link kernels (jfof_set_cta_shape), each
   NULL = the context's; per-box choices come from jfof_autotune.  use_graph != 0: the first call captures every box's
   pipeline as a parallel branch of one CUDA graph and later calls with the
   same configuration (pointers, sizes, parameters, stream) replay it with a
   single launch; use_graph = 0 enqueues the boxes one after another (the
   per-box loop).  Capturing requires that the context's stream is not itself
   being captured. */
int jfof_fof_batched(jfof_ctx *ctx, const float *pos, const int64_t *h_box_offset, int32_t B,
                     const float *h_L, const float *h_b, const int32_t *h_n_axis,
                     const int32_t *h_small, const int32_t *h_dense, const int32_t *h_shape,
                     uint32_t flags, int32_t min_size, void *ws, size_t ws_bytes, int32_t *label,
                     int32_t *halo_id, int32_t *n_halos, int32_t use_graph);

/* Autotuner: times the a1-a7 pipeline on one box for candidate grids (the
   default n and n scaled by 0.8 and 1.26, where the workspace fits) and six
   cell-class pairs ((16, the default dense threshold), (8, 96), (16, 96),
   (16, 128), (16, 160), (24, 128)) with the default CTA shape, then the other CTA shapes for
   the best of those, `reps` runs each after a warm-up, and returns the
   fastest choice (*best_n_axis, *best_small, *best_dense, *best_shape) and
   its time in ms.  The choice is kept in the context by size bucket
   (round(2 log2 N), round(4 log2(L/b))); use_cache != 0 returns a kept choice
   for the same bucket without timing.  flush (device, may be NULL): a buffer
   larger than L2 that is overwritten before every timed run, so that boxes
   smaller than L2 are timed with their data in DRAM, as inside a batch.
   Synchronises.  Outputs label/halo_id [N] and n_halos [1] are scratch for
   the trials.  Labels never depend on the choice. */
int jfof_autotune(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, uint32_t flags,
                  int32_t min_size, void *ws, size_t ws_bytes, int32_t *label, int32_t *halo_id,
                  int32_t *n_halos, int32_t reps, int32_t use_cache, void *flush, size_t flush_bytes,
                  int32_t *best_n_axis, int32_t *best_small, int32_t *best_dense, int32_t *best_shape,
                  float *best_ms);

/* Convenience: a1-a7 in one call (bin, link, groups) with one workspace. */
int jfof_fof_all_bytes(int64_t N, int32_t n_axis, size_t *bytes);
int jfof_fof(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, int32_t n_axis,
             uint32_t flags, int32_t min_size, void *ws, size_t ws_bytes, int32_t *label,
             int32_t *halo_id, int32_t *count, int32_t *halo_start, int32_t *members,
             int32_t *n_halos);

/* One step of the whole plain path (Sec. 2 steps (i)-(vi) and Sec. 3.1,
   Eq. 4: a1-a8) from HOST buffers.  h_pos / h_vel: host float32 [N,3]
   (h_vel may be NULL: no velocity outputs); page-locked memory (cudaHostAlloc
   or cudaHostRegister) lets the uploads run asynchronously, pageable memory
   works but the copies then block the caller.  d_pos / d_vel: the caller's
   device staging buffers [N,3] (d_vel NULL iff h_vel is NULL); they receive
   the uploaded inputs and stay valid afterwards.  Positions are uploaded on
   the context's stream; velocities on a library-owned copy stream after the
   positions, so their upload overlaps the FoF kernels; the halo properties
   and everything later enqueued on the context's stream wait for it.  Then
   exactly jfof_fof (ws of jfof_fof_all_bytes(N, n) bytes) and
   jfof_halo_props with H_cap = max(1, N / min_size), with the same outputs
   and the same errors; host buffers must stay unchanged until the context's
   stream has passed this call.  Argument errors return before any copy. */
int jfof_fof_host(jfof_ctx *ctx, const float *h_pos, const float *h_vel, int64_t N, float L, float b,
                  int32_t n_axis, uint32_t flags, int32_t min_size, float particle_mass, float *d_pos,
                  float *d_vel, void *ws, size_t ws_bytes, int32_t *label, int32_t *halo_id,
                  int32_t *count, int32_t *halo_start, int32_t *members, int32_t *n_halos,
                  float *mass, float *com, float *vmean, float *sigv);

/* ---------------------------------------------------------------------- */
/* Sub-halos (Sec. 2.1.1, Eq. 3): a second FoF pass inside each halo in     */
/* phase space.  Members i, j of one halo are friends when                  */
/*   |x_i - x_j|^2 / sigma_x + |v_i - v_j|^2 / sigma_v <= 1                  */
/* (minimum-image dx), evaluated in binary32 as dxx = (dx*dx + dy*dy) +      */
/* dz*dz, dvv likewise, link iff dxx*f32(1/sigma_x) + dvv*f32(1/sigma_v) <=   */
/* 1, each operation rounded once (sigma = +inf switches its term off).      */

/* Workspace bytes for jfof_subhalos (member-ordered positions, velocities  */
/* and a forest over member slots: 36 B per particle). */
int jfof_subhalos_bytes(int64_t N, size_t *bytes);

/* sub_label[N] (device int32): for a member of a halo, the smallest index   */
/* of its phase-space group inside that halo; for a particle outside every   */
/* halo, its own index.  pos, vel float32 [N,3] (JFOF_WRAP as jfof_fof);     */
/* halo_start/members/n_halos: the CSR of jfof_groups or jfof_fof.  Feeding  */
/* sub_label to jfof_groups gives sub-halo ids and sizes.  Each halo's pairs */
/* are all tested (cost grows with the square of the halo size). */
int jfof_subhalos(jfof_ctx *ctx, const float *pos, const float *vel, int64_t N, float L,
                  uint32_t flags, const int32_t *halo_start, const int32_t *members,
                  const int32_t *n_halos, int64_t H_cap, float sigma_x, float sigma_v, void *ws,
                  size_t ws_bytes, int32_t *sub_label);

/* ---------------------------------------------------------------------- */
/* Decorated frozen assignment (Sec. 3.1.1, Eq. 5) and the soft mass        */
/* function.  The decoration is the particle standard deviation about the   */
/* halo centre, D_h = sqrt(sum_i |mi(x_i - X_h)|^2 / (3 n_h)), an analytic   */
/* function of the positions used as a proxy for the halo mass (the paper's */
/* sigma, which falls as the mass grows).  The soft mass function bins the  */
/* log-masses ell_h = log(particle_mass n_h) with logistic edges: bin k      */
/* gets S((ell_h - e_k)/w) - S((ell_h - e_{k+1})/w), S(t) = 1/(1 + exp(-t)). */
/* Its gradient reaches the positions through the decoration: the decorated */
/* log-mass moves as -kappa log D_h (reading of Eq. 5 with sigma as an      */
/* inverse proxy), so g_D = -kappa g_ell / D, then the decoration's adjoint. */
/* Memberships are frozen; results are deterministic run to run.            */

/* D_h for h < *n_halos (device): pos float32 [N,3] (JFOF_WRAP as in         */
/* jfof_halo_props), the CSR of jfof_groups, com [H_cap,3] from               */
/* jfof_halo_props.  Writes dsig[H_cap] (entries below *n_halos). */
int jfof_halo_decoration(jfof_ctx *ctx, const float *pos, int64_t N, float L, uint32_t flags,
                         const int32_t *halo_start, const int32_t *members, const int32_t *n_halos,
                         int64_t H_cap, const float *com, float *dsig);

/* Its adjoint: g_pos[i] = g_dsig[h] mi(x_i - X_h) / (3 n_h D_h) for members */
/* of halo h (0 when D_h = 0), 0 for particles outside halos (halo_id = -1);  */
/* count [H] are the halo sizes.  g_pos float32 [N,3] (device). */
int jfof_halo_decoration_backward(jfof_ctx *ctx, const float *pos, const int32_t *halo_id,
                                  const int32_t *count, int64_t N, float L, uint32_t flags,
                                  const float *com, const float *dsig, const float *g_dsig,
                                  float *g_pos);

/* Workspace bytes of jfof_soft_hmf for up to H_cap halos and B bins          */
/* (1 <= B <= 4096). */
int jfof_soft_hmf_bytes(int64_t H_cap, int32_t B, size_t *bytes);

/* Soft mass function: hist[k], k < B, over edges[0..B] (device float32,      */
/* ascending log-mass) with softness width > 0, from the halo sizes count    */
/* [*n_halos] (device). */
int jfof_soft_hmf(jfof_ctx *ctx, const int32_t *count, const int32_t *n_halos, int64_t H_cap,
                  float particle_mass, const float *edges, int32_t B, float width, void *ws,
                  size_t ws_bytes, float *hist);

/* Its vector-Jacobian product to the decoration: g_dsig[h] = -kappa g_ell_h  */
/* / D_h, g_ell_h = sum_k g_hist[k] (S'(a_k) - S'(a_{k+1})) / w, a_k =        */
/* (ell_h - e_k)/w (0 when D_h = 0).  g_dsig [H_cap] (device). */
int jfof_soft_hmf_backward(jfof_ctx *ctx, const int32_t *count, const int32_t *n_halos, int64_t H_cap,
                           float particle_mass, const float *dsig, const float *edges, int32_t B,
                           float width, float kappa, const float *g_hist, float *g_dsig);

/* ---------------------------------------------------------------------- */
/* Slabs: streaming FoF with bounded device memory (Sec. 2.2, streaming     */
/* mode) and the slab decomposition with union-find fusion of Sec. 2.3.     */
/*                                                                          */
/* The cell grid (n cells per axis, n >= 3) is cut into n_slabs slabs of    */
/* whole z-layers: slab s owns layers [n s / n_slabs, n (s+1) / n_slabs).    */
/* A slab's subset is its particles plus those of one more layer on each    */
/* side (periodic).  Cells are at least 1.01 b wide, so the subset holds    */
/* every friend of the slab's own particles; linking it in the full         */
/* periodic box finds only true links, and every link has an end in some    */
/* slab.  Fusing the slabs' components through the particles that two      */
/* subsets share gives exactly the FoF groups.  The z layer of a particle   */
/* is floor(z * f32(n/L)) clamped to [0, n-1], as on the device.            */

/* Host only (no GPU needed).  The subset of slab `slab` of n_slabs:        */
/* h_pos: HOST float32 [N,3] in [0, L) (JFOF_ERANGE otherwise); n_axis =    */
/* cells per axis (0 = the default for N, as jfof_fof).  Writes to HOST      */
/* h_idx[n_sel] the subset's global indices in ascending order and to        */
/* h_core[n_sel] 1 for the slab's own particles, 0 for the extra layers;    */
/* either may be NULL (count only).  *n_sel = subset size.  JFOF_EINVAL if   */
/* n < 3, n_slabs < 1, n_slabs > n or slab is out of range. */
int jfof_slab_select(const float *h_pos, int64_t N, float L, float b, int32_t n_axis,
                     int32_t n_slabs, int32_t slab, int64_t *h_idx, uint8_t *h_core,
                     int64_t *n_sel);

/* Host only.  The union-find fusion of Sec. 2.3 over global indices:       */
/* classes of [0, N) joined pairwise by (h_a[k], h_b[k]), k < n_pairs (HOST  */
/* int32), with the smaller index as root; h_label[i] = root of h_pre[i]'s   */
/* class (HOST int32 [N] in and out; h_pre entries in [0, N)).  With         */
/* h_pre[i] = particle i's label in its own slab and one pair per particle   */
/* of an extra layer (its label in its own slab, its label in the other     */
/* slab), h_label is the smallest index of each FoF group. */
int jfof_merge_labels(int64_t N, const int32_t *h_pre, int64_t n_pairs, const int32_t *h_a,
                      const int32_t *h_b, int32_t *h_label);

/* Device workspace bytes for jfof_fof_stream: the largest slab subset's     */
/* positions, labels and bin/link workspace (reads HOST h_pos to size the    */
/* subsets). */
int jfof_fof_stream_bytes(const float *h_pos, int64_t N, float L, float b, int32_t n_axis,
                          int32_t n_slabs, size_t *bytes);

/* FoF of a box whose positions stay in HOST memory (h_pos, float32 [N,3] in */
/* [0, L)), slab by slab on the device: each subset is gathered on the host, */
/* uploaded into ws, binned and linked (the kernels of jfof_bin_cells and    */
/* jfof_link on the same grid), and its labels copied back; the slabs are   */
/* then fused as jfof_merge_labels describes.  Device memory is bounded by   */
/* the largest subset (jfof_fof_stream_bytes) instead of the whole box.      */
/* Outputs (HOST): h_label[N] raw labels (smallest index of the group),      */
/* h_halo_id[N] (ascending with the raw label, -1 below min_size; may be     */
/* NULL), *n_halos (may be NULL).  Synchronises the context's stream once    */
/* per slab; device errors are returned directly.  Equal to jfof_fof's      */
/* labels and halo ids for every n_slabs. */
int jfof_fof_stream(jfof_ctx *ctx, const float *h_pos, int64_t N, float L, float b,
                    int32_t n_axis, int32_t n_slabs, int32_t min_size, void *ws, size_t ws_bytes,
                    int32_t *h_label, int32_t *h_halo_id, int64_t *n_halos);

/* ---------------------------------------------------------------------- */
/* No-allocation variant (the paper has no counterpart).                   */

/* jfof_fof without a workspace argument, for callers that must not allocate
   device memory: e.g. an in-situ analysis hook inside a simulation or
   framework that owns all device memory through its own pool, or a
   latency-critical path that cannot afford the implicit device-wide
   synchronisation cudaMalloc/cudaFree may perform.  Inputs and outputs are
   the caller's, exactly as for jfof_fof (same results).  The scratch is a
   fixed 16 MiB device array inside the library, present on every GPU that
   loads it until the process exits; the call allocates nothing.
   Limit: jfof_fof_all_bytes(N, n_axis) must not exceed 16 MiB (about
   1.9e5 particles at the default grid); larger inputs return JFOF_ENOMEM
   before any work is enqueued.
   The first call on a device looks up the array's device address with that
   device current (a synchronous runtime call); make that first call before
   any stream capture.  All calls share the one array: calls whose work
   overlaps on the same GPU race on it, so the caller must serialise them
   (one stream, or events).  Each call initialises all the scratch it reads. */
int jfof_fof_static(jfof_ctx *ctx, const float *pos, int64_t N, float L, float b, int32_t n_axis,
                    uint32_t flags, int32_t min_size, int32_t *label, int32_t *halo_id,
                    int32_t *count, int32_t *halo_start, int32_t *members, int32_t *n_halos);

#ifdef __cplusplus
}
#endif
#endif /* JFOF_H */
