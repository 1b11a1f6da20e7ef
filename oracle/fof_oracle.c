/*
 * fof_oracle.c -- plain, slow CPU oracle for the Friends-of-Friends hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the CUDA
 * library; each side implements the method from the paper independently.
 *
 * Build with  -O2 -ffp-contract=off  and no fast-math: every float operation
 * below must be one IEEE binary32 operation, rounded once, so that the pair
 * predicate is evaluated exactly as specified (no fused multiply-add).
 *
 * What it computes, and where the paper defines it (Horowitz & Bayer,
 * "jFoF: GPU Cluster Finding with Gradient Propagation"):
 *   - FoF groups: two particles are friends when their (periodic minimum-image)
 *     separation is within the linking length b; groups are the connected
 *     components of the friendship graph (Sec. 1; Sec. 2 steps (iv)-(v);
 *     Algorithm 2 uses "<= b").  Raw label = smallest particle index in the
 *     component, i.e. the fixed point of the min-label propagation of Sec. 2
 *     step (v) and Algorithm 2.
 *   - candidate search on a linked-cell grid over the periodic box, 27-cell
 *     stencil with (. mod n) wrapping (Sec. 2.2, Algorithm 2); uncapped.
 *   - compaction to 0..H-1 and per-group counts (Sec. 2 step (vi)), with a
 *     minimum group size cut.
 *   - halo properties: mass, periodic centre of mass, velocity mean and 1-D
 *     velocity dispersion (Sec. 3.1, Eq. 4, Table 1 "halo position").
 *   - frozen-assignment adjoint of those properties (Sec. 3.1, Eq. 4).
 *   - REINFORCE topological mode: Bernoulli edges over a fixed candidate list
 *     (Sec. 3.2, Eq. 8; neighbour list not rebuilt), per-sample FoF, and the
 *     score-function gradient estimate with a baseline (Eqs. 6-7).
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   - link iff d2 <= b2, d2 = (dx*dx + dy*dy) + dz*dz in binary32, with the
 *     minimum-image correction applied per axis to dx = xj - xi:
 *       if dx > L/2: dx -= L; else if dx < -L/2: dx += L.
 *   - cell grid: n <= floor(L / (1.01 b)) cells per axis (the printed
 *     n = ceil(L/b) gives cells smaller than b and misses links); n = 1 or
 *     n >= 3; labels do not depend on n.
 *   - optional wrap x' = x - L*floor(x/L), then x' >= L or x' < 0 -> 0.
 *   - halo ids ascending by raw label; groups with count >= min_size kept.
 *   - periodic COM about the group's smallest-index member r:
 *       com = wrap(x_r + (1/n) sum_i mi(x_i - x_r)).
 *   - velocity dispersion sigma^2 = (1/(3n)) sum_i |v_i - vbar|^2 (two-pass).
 *   - REINFORCE edge probability p = 1/(1+E(-z)), z = (b-d)/tau (form 0) or
 *     z = alpha (b2 - d2)/b2 (form 1, Eq. 8); candidates d2 < (1.5 b)^2 style
 *     cut r_cut; E is the Cody-Waite + degree-7 Taylor exponential below;
 *     uniforms from Philox4x32-10 (Salmon et al., SC'11) keyed by the seed with
 *     counter (min index, max index, floor(k/4), 0), word k mod 4, top 24 bits.
 *
 * Parity pins (see tests/): brute force for small N, cubic lattices, chains
 * across the periodic boundary, exact ties, invariants, closed-form halos,
 * central finite differences, Philox known-answer vectors, exact enumeration
 * of tiny REINFORCE graphs.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Status codes (own numbering; the oracle reports, it never aborts).        */
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ERANGE 2
#define ORC_ENOMEM 3

/* ------------------------------------------------------------------------ */
/* The pair predicate (Sec. 2 step (iv); Algorithm 2 minimum image).          */

static float orc_min_image(float xj, float xi, float L, float hL)
{
    float d = xj - xi;
    if (d > hL)
        d = d - L;
    else if (d < -hL)
        d = d + L;
    return d;
}

/* d2 between particles i and j (float positions, AoS [N,3]). */
float orc_dist2(const float *pi, const float *pj, float L)
{
    float hL = 0.5f * L;
    float dx = orc_min_image(pj[0], pi[0], L, hL);
    float dy = orc_min_image(pj[1], pi[1], L, hL);
    float dz = orc_min_image(pj[2], pi[2], L, hL);
    float sx = dx * dx;
    float sy = dy * dy;
    float sz = dz * dz;
    float s = sx + sy;
    return s + sz;
}

/* ------------------------------------------------------------------------ */
/* Union-find with the smaller index as the root (sequential).               */

static int32_t uf_find(int32_t *parent, int32_t x)
{
    int32_t r = x;
    while (parent[r] != r)
        r = parent[r];
    while (parent[x] != r) { /* path compression */
        int32_t nx = parent[x];
        parent[x] = r;
        x = nx;
    }
    return r;
}

static void uf_union(int32_t *parent, int32_t a, int32_t b)
{
    int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb)
        return;
    if (ra < rb)
        parent[rb] = ra;
    else
        parent[ra] = rb;
}

/* ------------------------------------------------------------------------ */
/* Input normalisation: optional periodic wrap (Algorithm 2 "X mod L").       */

int orc_wrap(float *pos, int64_t N, float L)
{
    for (int64_t i = 0; i < 3 * N; ++i) {
        float x = pos[i];
        float q = floorf(x / L);
        float w = x - L * q;
        if (w >= L)
            w = 0.0f;
        if (w < 0.0f)
            w = 0.0f;
        pos[i] = w;
    }
    return ORC_OK;
}

/* Largest legal cells-per-axis for the grid: floor(L / (1.01 b)); n = 2 is
   replaced by 1 so that the 27-cell stencil never visits a cell twice. */
int32_t orc_max_cells_per_axis(float L, float b)
{
    double m = floor((double)L / (1.01 * (double)b));
    if (m < 1.0)
        m = 1.0;
    if (m > 2048.0)
        m = 2048.0;
    int32_t n = (int32_t)m;
    if (n == 2)
        n = 1;
    return n;
}

static int32_t cell_coord(float x, float inv_cell, int32_t n)
{
    float u = x * inv_cell;
    int32_t c = (int32_t)floorf(u);
    if (c > n - 1)
        c = n - 1;
    if (c < 0)
        c = 0;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Cell list: particles counting-sorted by cell id c = ix + n(iy + n iz), with */
/* their positions copied in that order so that a cell is one contiguous run. */

typedef struct {
    int32_t n;
    int64_t ncell;
    int64_t *start;  /* [ncell + 1] */
    int32_t *idx;    /* [N] original index, cell order, ascending within a cell */
    float *cpos;     /* [3N] positions in cell order */
} cell_list;

static void cell_list_free(cell_list *cl)
{
    free(cl->start);
    free(cl->idx);
    free(cl->cpos);
}

static int cell_list_build(cell_list *cl, const float *pos, int64_t N, float L, int32_t n)
{
    cl->n = n;
    cl->ncell = (int64_t)n * n * n;
    cl->start = (int64_t *)calloc((size_t)cl->ncell + 1, sizeof(int64_t));
    cl->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    cl->cpos = (float *)malloc(sizeof(float) * 3 * (size_t)N);
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!cl->start || !cl->idx || !cl->cpos || !cid) {
        free(cid);
        cell_list_free(cl);
        return ORC_ENOMEM;
    }
    float inv_cell = (float)((double)n / (double)L);
    for (int64_t i = 0; i < N; ++i) {
        int32_t ix = cell_coord(pos[3 * i + 0], inv_cell, n);
        int32_t iy = cell_coord(pos[3 * i + 1], inv_cell, n);
        int32_t iz = cell_coord(pos[3 * i + 2], inv_cell, n);
        cid[i] = ix + (int64_t)n * (iy + (int64_t)n * iz);
        cl->start[cid[i] + 1] += 1;
    }
    for (int64_t c = 0; c < cl->ncell; ++c)
        cl->start[c + 1] += cl->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)cl->ncell);
    if (!fill) {
        free(cid);
        cell_list_free(cl);
        return ORC_ENOMEM;
    }
    memcpy(fill, cl->start, sizeof(int64_t) * (size_t)cl->ncell);
    for (int64_t i = 0; i < N; ++i) { /* ascending i: stable within a cell */
        int64_t k = fill[cid[i]]++;
        cl->idx[k] = (int32_t)i;
        cl->cpos[3 * k + 0] = pos[3 * i + 0];
        cl->cpos[3 * k + 1] = pos[3 * i + 1];
        cl->cpos[3 * k + 2] = pos[3 * i + 2];
    }
    free(fill);
    free(cid);
    return ORC_OK;
}

/* The distinct cells among the 27 neighbours (. mod n) of cell (ix,iy,iz). */
static int neighbour_cells(const cell_list *cl, int64_t c, int64_t out[27])
{
    int32_t n = cl->n;
    int32_t ix = (int32_t)(c % n), iy = (int32_t)((c / n) % n), iz = (int32_t)(c / ((int64_t)n * n));
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int32_t cx = ((ix + dx) % n + n) % n;
                int32_t cy = ((iy + dy) % n + n) % n;
                int32_t cz = ((iz + dz) % n + n) % n;
                int64_t nc = cx + (int64_t)n * (cy + (int64_t)n * cz);
                int dup = 0;
                for (int s = 0; s < cnt; ++s)
                    if (out[s] == nc)
                        dup = 1;
                if (!dup)
                    out[cnt++] = nc;
            }
    return cnt;
}

/* Default grid for the oracle: the largest legal n with n^3 <= 16 N. */
static int32_t oracle_grid(int64_t N, float L, float b)
{
    int32_t n = orc_max_cells_per_axis(L, b);
    while (n > 3 && (double)n * n * n > 16.0 * (double)N)
        --n;
    return n;
}

/* ------------------------------------------------------------------------ */
/* FoF labels via a linked-cell grid + union-find (Sec. 2.2, Algorithm 2).    */
/* label[i] = smallest index in i's component.  n_axis = 0 picks a default    */
/* grid.  Every pair (i, j), i < j, in the same or adjacent cells is tested   */
/* once.  Returns ORC_* status.                                               */

int orc_fof_labels(const float *pos, int64_t N, float L, float b, int32_t n_axis,
                   int32_t *label)
{
    if (N < 1 || !(L > 0.0f) || !(b > 0.0f) || !(b < 0.5f * L))
        return ORC_EINVAL;
    for (int64_t i = 0; i < 3 * N; ++i)
        if (!(pos[i] >= 0.0f && pos[i] < L))
            return ORC_ERANGE;
    int32_t nmax = orc_max_cells_per_axis(L, b);
    int32_t n = n_axis > 0 ? n_axis : oracle_grid(N, L, b);
    if (n > nmax || n == 2)
        return ORC_EINVAL;
    cell_list cl;
    int st = cell_list_build(&cl, pos, N, L, n);
    if (st != ORC_OK)
        return st;
    int32_t *parent = label; /* union-find forest lives in the output */
    for (int64_t i = 0; i < N; ++i)
        parent[i] = (int32_t)i;
    float b2 = b * b;
    for (int64_t c = 0; c < cl.ncell; ++c) {
        if (cl.start[c] == cl.start[c + 1])
            continue;
        int64_t nb[27];
        int nnb = neighbour_cells(&cl, c, nb);
        for (int64_t a = cl.start[c]; a < cl.start[c + 1]; ++a) {
            int32_t i = cl.idx[a];
            for (int s = 0; s < nnb; ++s)
                for (int64_t k = cl.start[nb[s]]; k < cl.start[nb[s] + 1]; ++k) {
                    int32_t j = cl.idx[k];
                    if (j <= i)
                        continue; /* each unordered pair once */
                    if (orc_dist2(cl.cpos + 3 * a, cl.cpos + 3 * k, L) <= b2)
                        uf_union(parent, i, j);
                }
        }
    }
    for (int64_t i = 0; i < N; ++i)
        label[i] = uf_find(parent, (int32_t)i);
    cell_list_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The same labels on T threads, for boxes too large for one core.           */
/*                                                                            */
/* The cells are cut into T slabs of whole z-layers; cells are numbered       */
/* z-major, so the particles of a slab are one contiguous run of cell-list    */
/* slots.  Thread t visits the pairs (i, j), i < j, whose particle i lies in  */
/* its slab -- the pairs orc_fof_labels tests from i's side, so every pair is */
/* tested exactly once -- with the same predicate.  A linked pair with both   */
/* slots in the slab is united at once in a forest over slots (the smaller    */
/* slot is the root, so thread t reads and writes only its own slots); a      */
/* linked pair with one slot in another slab is recorded.  The recorded pairs */
/* are then united one after another in thread order.  Both sides unite       */
/* exactly the linked pairs, so the components equal those of the sequential  */
/* union-find, and label[i] = smallest original index in i's component        */
/* (Sec. 2 step (v)) is the same.  This is the slab decomposition with        */
/* union-find fusion of Sec. 2.3, with threads in place of devices.           */


typedef struct {
    const float *pos;
    const cell_list *cl;
    int64_t lo, hi;      /* work range of a parallel phase */
    float inv_cell;
    int64_t *cid;
    int32_t *parent;
    int32_t *root;
    int32_t *minidx;
    int32_t *label;
    int64_t *fill;
    /* linking */
    float L, b2;
    int64_t s0, s1;      /* slots of the slab */
    int64_t *cross;      /* recorded pairs of slots (a, k) */
    int64_t ncross, capcross;
    int status;
} mt_job;

static void mt_run(mt_job *jobs, int T, void *(*fn)(void *))
{
    pthread_t th[256];
    int started[256];
    for (int t = 0; t < T; ++t)
        started[t] = pthread_create(&th[t], NULL, fn, &jobs[t]) == 0;
    for (int t = 0; t < T; ++t) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            fn(&jobs[t]); /* no thread: run the share here */
    }
}

static void *mt_cell_ids(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    int32_t n = jb->cl->n;
    for (int64_t i = jb->lo; i < jb->hi; ++i) {
        int32_t ix = cell_coord(jb->pos[3 * i + 0], jb->inv_cell, n);
        int32_t iy = cell_coord(jb->pos[3 * i + 1], jb->inv_cell, n);
        int32_t iz = cell_coord(jb->pos[3 * i + 2], jb->inv_cell, n);
        jb->cid[i] = ix + (int64_t)n * (iy + (int64_t)n * iz);
        __atomic_fetch_add(&jb->cl->start[jb->cid[i] + 1], 1, __ATOMIC_RELAXED);
    }
    return NULL;
}

static void *mt_fill(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    const cell_list *cl = jb->cl;
    for (int64_t i = jb->lo; i < jb->hi; ++i) {
        int64_t k = __atomic_fetch_add(&jb->fill[jb->cid[i]], 1, __ATOMIC_RELAXED);
        cl->idx[k] = (int32_t)i;
        cl->cpos[3 * k + 0] = jb->pos[3 * i + 0];
        cl->cpos[3 * k + 1] = jb->pos[3 * i + 1];
        cl->cpos[3 * k + 2] = jb->pos[3 * i + 2];
    }
    return NULL;
}

static int mt_record(mt_job *jb, int64_t a, int64_t k)
{
    if (jb->ncross == jb->capcross) {
        int64_t cap = jb->capcross ? 2 * jb->capcross : 4096;
        int64_t *p = (int64_t *)realloc(jb->cross, sizeof(int64_t) * 2 * (size_t)cap);
        if (!p)
            return ORC_ENOMEM;
        jb->cross = p;
        jb->capcross = cap;
    }
    jb->cross[2 * jb->ncross] = a;
    jb->cross[2 * jb->ncross + 1] = k;
    jb->ncross += 1;
    return ORC_OK;
}

static void *mt_link_slab(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    const cell_list *cl = jb->cl;
    for (int64_t c = jb->lo; c < jb->hi && jb->status == ORC_OK; ++c) {
        if (cl->start[c] == cl->start[c + 1])
            continue;
        int64_t nb[27];
        int nnb = neighbour_cells(cl, c, nb);
        for (int64_t a = cl->start[c]; a < cl->start[c + 1]; ++a) {
            int32_t i = cl->idx[a];
            for (int s = 0; s < nnb; ++s)
                for (int64_t k = cl->start[nb[s]]; k < cl->start[nb[s] + 1]; ++k) {
                    if (cl->idx[k] <= i)
                        continue; /* each unordered pair once, from its smaller index */
                    if (!(orc_dist2(cl->cpos + 3 * a, cl->cpos + 3 * k, jb->L) <= jb->b2))
                        continue;
                    if (k >= jb->s0 && k < jb->s1)
                        uf_union(jb->parent, (int32_t)a, (int32_t)k);
                    else if (mt_record(jb, a, k) != ORC_OK)
                        jb->status = ORC_ENOMEM;
                }
        }
    }
    return NULL;
}

/* root of each slot, with no writes (the forest is complete) */
static void *mt_roots(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    for (int64_t a = jb->lo; a < jb->hi; ++a) {
        int32_t r = (int32_t)a;
        while (jb->parent[r] != r)
            r = jb->parent[r];
        jb->root[a] = r;
    }
    return NULL;
}

/* smallest original index per root */
static void *mt_minidx(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    for (int64_t a = jb->lo; a < jb->hi; ++a) {
        int32_t *m = &jb->minidx[jb->root[a]], v = jb->cl->idx[a];
        int32_t cur = __atomic_load_n(m, __ATOMIC_RELAXED);
        while (v < cur && !__atomic_compare_exchange_n(m, &cur, v, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED))
            ;
    }
    return NULL;
}

static void *mt_labels(void *arg)
{
    mt_job *jb = (mt_job *)arg;
    for (int64_t a = jb->lo; a < jb->hi; ++a)
        jb->label[jb->cl->idx[a]] = jb->minidx[jb->root[a]];
    return NULL;
}

static void mt_split(mt_job *jobs, int T, int64_t total)
{
    for (int t = 0; t < T; ++t) {
        jobs[t].lo = total * t / T;
        jobs[t].hi = total * (t + 1) / T;
    }
}

int orc_fof_labels_mt(const float *pos, int64_t N, float L, float b, int32_t n_axis,
                      int32_t nthreads, int32_t *label)
{
    if (N < 1 || !(L > 0.0f) || !(b > 0.0f) || !(b < 0.5f * L) || nthreads < 1)
        return ORC_EINVAL;
    for (int64_t i = 0; i < 3 * N; ++i)
        if (!(pos[i] >= 0.0f && pos[i] < L))
            return ORC_ERANGE;
    int32_t nmax = orc_max_cells_per_axis(L, b);
    int32_t n = n_axis > 0 ? n_axis : oracle_grid(N, L, b);
    if (n > nmax || n == 2)
        return ORC_EINVAL;
    int T = nthreads > 256 ? 256 : nthreads;
    cell_list cl;
    cl.n = n;
    cl.ncell = (int64_t)n * n * n;
    cl.start = (int64_t *)calloc((size_t)cl.ncell + 1, sizeof(int64_t));
    cl.idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    cl.cpos = (float *)malloc(sizeof(float) * 3 * (size_t)N);
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    mt_job *jobs = (mt_job *)calloc((size_t)T, sizeof(mt_job));
    int32_t *parent = NULL, *root = NULL, *minidx = NULL;
    int64_t *fill = NULL;
    int st = ORC_ENOMEM;
    if (!cl.start || !cl.idx || !cl.cpos || !cid || !jobs)
        goto done;
    for (int t = 0; t < T; ++t) {
        jobs[t].pos = pos;
        jobs[t].cl = &cl;
        jobs[t].inv_cell = (float)((double)n / (double)L);
        jobs[t].cid = cid;
        jobs[t].L = L;
        jobs[t].b2 = b * b;
    }
    /* cell list: counts, offsets, then slots (order inside a cell is free) */
    mt_split(jobs, T, N);
    mt_run(jobs, T, mt_cell_ids);
    for (int64_t c = 0; c < cl.ncell; ++c)
        cl.start[c + 1] += cl.start[c];
    fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)cl.ncell);
    if (!fill)
        goto done;
    memcpy(fill, cl.start, sizeof(int64_t) * (size_t)cl.ncell);
    for (int t = 0; t < T; ++t)
        jobs[t].fill = fill;
    mt_run(jobs, T, mt_fill);
    free(fill);
    fill = NULL;
    free(cid);
    cid = NULL;
    /* slabs of z-layers, linked in parallel */
    parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!parent)
        goto done;
    for (int64_t a = 0; a < N; ++a)
        parent[a] = (int32_t)a;
    int64_t layer = (int64_t)n * n;
    for (int t = 0; t < T; ++t) {
        int64_t z0 = (int64_t)n * t / T, z1 = (int64_t)n * (t + 1) / T;
        jobs[t].lo = z0 * layer;
        jobs[t].hi = z1 * layer;
        jobs[t].s0 = cl.start[z0 * layer];
        jobs[t].s1 = cl.start[z1 * layer];
        jobs[t].parent = parent;
        jobs[t].status = ORC_OK;
    }
    mt_run(jobs, T, mt_link_slab);
    for (int t = 0; t < T; ++t)
        if (jobs[t].status != ORC_OK)
            goto done;
    /* pairs across slabs, one after another */
    for (int t = 0; t < T; ++t)
        for (int64_t e = 0; e < jobs[t].ncross; ++e)
            uf_union(parent, (int32_t)jobs[t].cross[2 * e], (int32_t)jobs[t].cross[2 * e + 1]);
    /* label = smallest original index of the component */
    root = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    minidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!root || !minidx)
        goto done;
    for (int64_t a = 0; a < N; ++a)
        minidx[a] = INT32_MAX;
    mt_split(jobs, T, N);
    for (int t = 0; t < T; ++t) {
        jobs[t].root = root;
        jobs[t].minidx = minidx;
        jobs[t].label = label;
    }
    mt_run(jobs, T, mt_roots);
    mt_run(jobs, T, mt_minidx);
    mt_run(jobs, T, mt_labels);
    st = ORC_OK;
done:
    if (jobs)
        for (int t = 0; t < T; ++t)
            free(jobs[t].cross);
    free(jobs);
    free(fill);
    free(cid);
    free(parent);
    free(root);
    free(minidx);
    cell_list_free(&cl);
    return st;
}

/* O(N^2) brute force over all pairs with the same predicate (pin for the
   cell-list oracle, Sec. 2: "the naive cost of pairwise searches"). */
int orc_fof_brute(const float *pos, int64_t N, float L, float b, int32_t *label)
{
    if (N < 1 || !(b > 0.0f) || !(b < 0.5f * L))
        return ORC_EINVAL;
    float b2 = b * b;
    for (int64_t i = 0; i < N; ++i)
        label[i] = (int32_t)i;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j)
            if (orc_dist2(pos + 3 * i, pos + 3 * j, L) <= b2)
                uf_union(label, (int32_t)i, (int32_t)j);
    for (int64_t i = 0; i < N; ++i)
        label[i] = uf_find(label, (int32_t)i);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Compaction + histogram + minimum-size cut (Sec. 2 step (vi); Alg. 1-2     */
/* "Compaction").  halo_id ascending by raw label; -1 below the cut.         */
/* count has room for N entries.  Returns H (>= 0) or -1 on bad input.       */

int64_t orc_groups(const int32_t *label, int64_t N, int32_t min_size,
                   int32_t *halo_id, int32_t *count)
{
    if (N < 1 || min_size < 1)
        return -1;
    int64_t *cnt = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    int64_t *hid = (int64_t *)malloc(sizeof(int64_t) * N);
    if (!cnt || !hid) {
        free(cnt);
        free(hid);
        return -1;
    }
    for (int64_t i = 0; i < N; ++i) {
        if (label[i] < 0 || label[i] >= N) {
            free(cnt);
            free(hid);
            return -1;
        }
        cnt[label[i]] += 1;
    }
    int64_t H = 0;
    for (int64_t r = 0; r < N; ++r) {
        hid[r] = -1;
        if (label[r] == r && cnt[r] >= min_size) {
            hid[r] = H;
            count[H] = (int32_t)cnt[r];
            ++H;
        }
    }
    for (int64_t i = 0; i < N; ++i)
        halo_id[i] = (int32_t)hid[label[i]];
    free(cnt);
    free(hid);
    return H;
}

/* ------------------------------------------------------------------------ */
/* Halo properties in FP64 (Sec. 3.1, Eq. 4; Table 1).                       */
/* pos, vel: [N,3] doubles (float inputs widen exactly).  Outputs [H] / [H,3].*/

static double wrap_f64(double c, double L)
{
    double w = c - L * floor(c / L);
    if (w >= L || w < 0.0)
        w = 0.0;
    return w;
}

static double mi_f64(double d, double L)
{
    if (d > 0.5 * L)
        d -= L;
    else if (d < -0.5 * L)
        d += L;
    return d;
}

int orc_halo_props(const double *pos, const double *vel, const int32_t *halo_id,
                   int64_t N, int64_t H, double L, double particle_mass,
                   double *mass, double *com, double *vmean, double *sigv)
{
    if (H < 0)
        return ORC_EINVAL;
    int64_t *n = (int64_t *)calloc((size_t)(H > 0 ? H : 1), sizeof(int64_t));
    int64_t *ref = (int64_t *)malloc(sizeof(int64_t) * (size_t)(H > 0 ? H : 1));
    double *sx = (double *)calloc((size_t)(H > 0 ? 3 * H : 1), sizeof(double));
    double *sv = (double *)calloc((size_t)(H > 0 ? 3 * H : 1), sizeof(double));
    double *s2 = (double *)calloc((size_t)(H > 0 ? H : 1), sizeof(double));
    if (!n || !ref || !sx || !sv || !s2) {
        free(n); free(ref); free(sx); free(sv); free(s2);
        return ORC_ENOMEM;
    }
    for (int64_t h = 0; h < H; ++h)
        ref[h] = -1;
    /* pass 1: reference member (smallest index), counts, sums */
    for (int64_t i = 0; i < N; ++i) {
        int32_t h = halo_id[i];
        if (h < 0)
            continue;
        if (ref[h] < 0)
            ref[h] = i;
        n[h] += 1;
    }
    for (int64_t i = 0; i < N; ++i) {
        int32_t h = halo_id[i];
        if (h < 0)
            continue;
        for (int a = 0; a < 3; ++a) {
            sx[3 * h + a] += mi_f64(pos[3 * i + a] - pos[3 * ref[h] + a], L);
            sv[3 * h + a] += vel[3 * i + a];
        }
    }
    for (int64_t h = 0; h < H; ++h) {
        double nh = (double)n[h];
        mass[h] = particle_mass * nh;
        for (int a = 0; a < 3; ++a) {
            com[3 * h + a] = wrap_f64(pos[3 * ref[h] + a] + sx[3 * h + a] / nh, L);
            vmean[3 * h + a] = sv[3 * h + a] / nh;
        }
    }
    /* pass 2: dispersion about the mean */
    for (int64_t i = 0; i < N; ++i) {
        int32_t h = halo_id[i];
        if (h < 0)
            continue;
        for (int a = 0; a < 3; ++a) {
            double d = vel[3 * i + a] - vmean[3 * h + a];
            s2[h] += d * d;
        }
    }
    for (int64_t h = 0; h < H; ++h)
        sigv[h] = sqrt(s2[h] / (3.0 * (double)n[h]));
    free(n); free(ref); free(sx); free(sv); free(s2);
    return ORC_OK;
}

/* Frozen-assignment adjoint (Sec. 3.1, Eq. 4): memberships fixed, so
     d com_h / d x_i   = I / n_h             (every member, reference included)
     d vbar_h / d v_i  = I / n_h
     d sigma_h / d v_i = (v_i - vbar_h) / (3 n_h sigma_h), 0 when sigma_h = 0.
   g_com, g_vmean: [H,3] or NULL; g_sigv: [H] or NULL.  Outputs [N,3]. */
int orc_halo_props_backward(const double *vel, const int32_t *halo_id, int64_t N,
                            int64_t H, const double *vmean, const double *sigv,
                            const double *g_com, const double *g_vmean,
                            const double *g_sigv, double *g_pos, double *g_vel)
{
    int64_t *n = (int64_t *)calloc((size_t)(H > 0 ? H : 1), sizeof(int64_t));
    if (!n)
        return ORC_ENOMEM;
    for (int64_t i = 0; i < N; ++i)
        if (halo_id[i] >= 0)
            n[halo_id[i]] += 1;
    for (int64_t i = 0; i < N; ++i) {
        int32_t h = halo_id[i];
        for (int a = 0; a < 3; ++a) {
            g_pos[3 * i + a] = 0.0;
            g_vel[3 * i + a] = 0.0;
        }
        if (h < 0)
            continue;
        double nh = (double)n[h];
        for (int a = 0; a < 3; ++a) {
            if (g_com)
                g_pos[3 * i + a] = g_com[3 * h + a] / nh;
            double gv = 0.0;
            if (g_vmean)
                gv += g_vmean[3 * h + a] / nh;
            if (g_sigv && sigv[h] > 0.0)
                gv += g_sigv[h] * (vel[3 * i + a] - vmean[3 * h + a]) / (3.0 * nh * sigv[h]);
            g_vel[3 * i + a] = gv;
        }
    }
    free(n);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sub-halos: a second FoF pass inside each halo in phase space (Sec. 2.1.1, */
/* Eq. 3): members i, j of one halo are friends when                         */
/*   |x_i - x_j|^2 / sigma_x + |v_i - v_j|^2 / sigma_v <= 1,                 */
/* with the minimum-image position difference.  Binary32, in this order and  */
/* with no fused operations (both sides evaluate it the same way):           */
/*   dxx = (dx*dx + dy*dy) + dz*dz,  dvv = (du*du + dv*dv) + dw*dw,          */
/*   link iff dxx * inv_sx + dvv * inv_sv <= 1,                               */
/* inv_sx = f32(1/sigma_x), inv_sv = f32(1/sigma_v) (0 switches a term off).  */
/* sub_label[i] = smallest index of i's phase-space group inside its halo;   */
/* a particle outside every halo (halo_id = -1) is its own group.            */

float orc_phase_d2(const float *pi, const float *pj, const float *vi, const float *vj, float L,
                   float inv_sx, float inv_sv)
{
    float hL = 0.5f * L;
    float dx = orc_min_image(pj[0], pi[0], L, hL);
    float dy = orc_min_image(pj[1], pi[1], L, hL);
    float dz = orc_min_image(pj[2], pi[2], L, hL);
    float du = vj[0] - vi[0];
    float dv = vj[1] - vi[1];
    float dw = vj[2] - vi[2];
    float sxx = dx * dx;
    float syy = dy * dy;
    float szz = dz * dz;
    float dxx = sxx + syy;
    dxx = dxx + szz;
    float suu = du * du;
    float svv = dv * dv;
    float sww = dw * dw;
    float dvv = suu + svv;
    dvv = dvv + sww;
    float a = dxx * inv_sx;
    float c = dvv * inv_sv;
    return a + c;
}

int orc_subhalo_labels(const float *pos, const float *vel, const int32_t *halo_id, int64_t N,
                       int64_t H, float L, float inv_sx, float inv_sv, int32_t *sub_label)
{
    int64_t *start = (int64_t *)calloc((size_t)H + 1, sizeof(int64_t));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!start || !mem) {
        free(start); free(mem);
        return ORC_ENOMEM;
    }
    /* members of each halo in ascending index */
    for (int64_t i = 0; i < N; ++i)
        if (halo_id[i] >= 0)
            start[halo_id[i] + 1] += 1;
    for (int64_t h = 0; h < H; ++h)
        start[h + 1] += start[h];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(H > 0 ? H : 1));
    if (!fill) {
        free(start); free(mem);
        return ORC_ENOMEM;
    }
    memcpy(fill, start, sizeof(int64_t) * (size_t)H);
    for (int64_t i = 0; i < N; ++i)
        if (halo_id[i] >= 0)
            mem[fill[halo_id[i]]++] = (int32_t)i;
    free(fill);
    for (int64_t i = 0; i < N; ++i)
        sub_label[i] = (int32_t)i;
    /* every pair of members of one halo, once; the smaller index is the root */
    for (int64_t h = 0; h < H; ++h)
        for (int64_t a = start[h]; a < start[h + 1]; ++a)
            for (int64_t c = a + 1; c < start[h + 1]; ++c) {
                int32_t i = mem[a], j = mem[c];
                if (orc_phase_d2(pos + 3 * i, pos + 3 * j, vel + 3 * i, vel + 3 * j, L, inv_sx, inv_sv) <= 1.0f)
                    uf_union(sub_label, i, j);
            }
    for (int64_t i = 0; i < N; ++i)
        sub_label[i] = uf_find(sub_label, (int32_t)i);
    free(start); free(mem);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Decorated frozen assignment (Sec. 3.1.1, Eq. 5): a halo "decoration" that  */
/* is an analytic function of the member positions, here the particle        */
/* standard deviation about the halo centre,                                 */
/*   D_h = sqrt( (1/(3 n_h)) sum_i |mi(x_i - X_h)|^2 ),                        */
/* with X_h the periodic centre of mass (as orc_halo_props), used as a        */
/* differentiable proxy for the halo mass.  Memberships are frozen.          */

int orc_halo_decoration(const double *pos, const int32_t *halo_id, int64_t N, int64_t H,
                        double L, const double *com, double *dsig)
{
    int64_t *n = (int64_t *)calloc((size_t)(H > 0 ? H : 1), sizeof(int64_t));
    double *s2 = (double *)calloc((size_t)(H > 0 ? H : 1), sizeof(double));
    if (!n || !s2) {
        free(n); free(s2);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < N; ++i) {
        int32_t h = halo_id[i];
        if (h < 0)
            continue;
        n[h] += 1;
        for (int a = 0; a < 3; ++a) {
            double d = mi_f64(pos[3 * i + a] - com[3 * h + a], L);
            s2[h] += d * d;
        }
    }
    for (int64_t h = 0; h < H; ++h)
        dsig[h] = sqrt(s2[h] / (3.0 * (double)n[h]));
    free(n); free(s2);
    return ORC_OK;
}

/* Its frozen-assignment adjoint: with d_i = mi(x_i - X_h) and sum_i d_i = 0
   (X_h is the members' mean), d D_h / d x_i = d_i / (3 n_h D_h), 0 when
   D_h = 0.  g_pos[i] = g_dsig[h] d D_h / d x_i, 0 outside halos. */
int orc_halo_decoration_backward(const double *pos, const int32_t *halo_id, int64_t N, int64_t H,
                                 double L, const double *com, const double *dsig,
                                 const double *g_dsig, double *g_pos)
{
    int64_t *n = (int64_t *)calloc((size_t)(H > 0 ? H : 1), sizeof(int64_t));
    if (!n)
        return ORC_ENOMEM;
    for (int64_t i = 0; i < N; ++i)
        if (halo_id[i] >= 0)
            n[halo_id[i]] += 1;
    for (int64_t i = 0; i < N; ++i) {
        int32_t h = halo_id[i];
        for (int a = 0; a < 3; ++a)
            g_pos[3 * i + a] = 0.0;
        if (h < 0 || !(dsig[h] > 0.0))
            continue;
        double c = g_dsig[h] / (3.0 * (double)n[h] * dsig[h]);
        for (int a = 0; a < 3; ++a)
            g_pos[3 * i + a] = c * mi_f64(pos[3 * i + a] - com[3 * h + a], L);
    }
    free(n);
    return ORC_OK;
}

/* Soft histogram (Sec. 3.1.1: a "soft" histogram so that derivatives flow
   between bins): bin k of B collects, from every halo h with log-mass
   ell_h, the weight S((ell_h - e_k)/w) - S((ell_h - e_{k+1})/w), S the
   logistic function, e[0..B] the bin edges, w > 0 the softness.  As w -> 0
   it becomes the ordinary histogram. */
static double logistic(double t)
{
    return 1.0 / (1.0 + exp(-t));
}

int orc_soft_hist(const double *ell, int64_t H, const double *edges, int32_t B, double w,
                  double *hist)
{
    if (B < 1 || !(w > 0.0))
        return ORC_EINVAL;
    for (int32_t k = 0; k < B; ++k) {
        double s = 0.0;
        for (int64_t h = 0; h < H; ++h)
            s += logistic((ell[h] - edges[k]) / w) - logistic((ell[h] - edges[k + 1]) / w);
        hist[k] = s;
    }
    return ORC_OK;
}

/* Its vector-Jacobian product: g_ell[h] = sum_k g_hist[k] (S'(a_k) - S'(a_{k+1})) / w,
   a_k = (ell_h - e_k)/w, S' = S (1 - S). */
int orc_soft_hist_backward(const double *ell, int64_t H, const double *edges, int32_t B, double w,
                           const double *g_hist, double *g_ell)
{
    if (B < 1 || !(w > 0.0))
        return ORC_EINVAL;
    for (int64_t h = 0; h < H; ++h) {
        double s = 0.0;
        for (int32_t k = 0; k < B; ++k) {
            double s0 = logistic((ell[h] - edges[k]) / w), s1 = logistic((ell[h] - edges[k + 1]) / w);
            s += g_hist[k] * (s0 * (1.0 - s0) - s1 * (1.0 - s1)) / w;
        }
        g_ell[h] = s;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror & Shaw,      */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Round function:   */
/* two 32x32->64 multiplies by M0, M1, xor with the key, word shuffle; key   */
/* bumped by the Weyl constants between rounds.                              */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1) for edge (i,j) and sample k: 24 top bits of one Philox
   word, exactly representable in binary32. */
float orc_edge_uniform(uint64_t seed, int32_t i, int32_t j, int32_t k)
{
    uint32_t lo = (uint32_t)(i < j ? i : j), hi = (uint32_t)(i < j ? j : i);
    uint32_t ctr[4] = {lo, hi, (uint32_t)k >> 2, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    uint32_t w = out[k & 3];
    return (float)(w >> 8) * (1.0f / 16777216.0f);
}

/* ------------------------------------------------------------------------ */
/* Deterministic binary32 exponential: Cody-Waite range reduction            */
/* x = k ln2 + r with ln2 split into a binary32 head and tail, then the      */
/* degree-7 Taylor polynomial sum_{m<=7} r^m/m! by Horner with fused         */
/* multiply-add (correctly rounded fmaf), then scaling by 2^k through the    */
/* exponent field.  Input clamped to [-87, 87].  Constants are computed here */
/* from their mathematical definitions in FP64 and rounded once.            */

float orc_exp(float x)
{
    const float l2e = (float)(1.0 / M_LN2);
    const float ln2_hi = (float)M_LN2;
    const float ln2_lo = (float)(M_LN2 - (double)ln2_hi);
    float c[8];
    double f = 1.0;
    for (int m = 0; m < 8; ++m) {
        if (m > 0)
            f *= (double)m;
        c[m] = (float)(1.0 / f);
    }
    if (x > 87.0f)
        x = 87.0f;
    if (x < -87.0f)
        x = -87.0f;
    if (x != x)
        x = 0.0f;
    float t = x * l2e;
    float k = rintf(t);
    float r = fmaf(-k, ln2_hi, x);
    r = fmaf(-k, ln2_lo, r);
    float p = c[7];
    for (int m = 6; m >= 0; --m)
        p = fmaf(p, r, c[m]);
    int32_t ki = (int32_t)k;
    uint32_t bits = (uint32_t)(ki + 127) << 23;
    float scale;
    memcpy(&scale, &bits, sizeof(scale));
    return p * scale;
}

/* Edge probability (Eq. 8 and the distance-sigmoid form). */
float orc_edge_prob(float d, float d2, float b, float b2, int32_t form, float coef)
{
    float z;
    if (form == 0)
        z = (b - d) * coef; /* coef = 1/tau */
    else
        z = (b2 - d2) * coef; /* coef = alpha / b2 */
    float e = orc_exp(-z);
    return 1.0f / (1.0f + e);
}

/* ------------------------------------------------------------------------ */
/* Candidate pair list for REINFORCE (fixed, "do not rebuild the neighbor    */
/* list", Sec. 3.2): unordered pairs i<j with d2 < rc2, sorted by (i, j),     */
/* with d = sqrtf(d2) and the edge probability.  Returns the number of pairs; */
/* writes at most cap of them.  Negative on bad input.                       */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_pairs(const float *pos, int64_t N, float L, float b, float r_cut,
                  int32_t form, float coef, int64_t cap, int32_t *pi, int32_t *pj,
                  float *pd, float *pp)
{
    if (N < 1 || !(r_cut > 0.0f) || !(r_cut < 0.5f * L))
        return -1;
    for (int64_t i = 0; i < 3 * N; ++i)
        if (!(pos[i] >= 0.0f && pos[i] < L))
            return -1;
    float rc2 = r_cut * r_cut;
    float b2 = b * b;
    cell_list cl;
    if (cell_list_build(&cl, pos, N, L, oracle_grid(N, L, r_cut)) != ORC_OK)
        return -1;
    int64_t *where = (int64_t *)malloc(sizeof(int64_t) * (size_t)N); /* slot of index i */
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!where || !buf) {
        free(where); free(buf); cell_list_free(&cl);
        return -1;
    }
    for (int64_t a = 0; a < N; ++a)
        where[cl.idx[a]] = a;
    int64_t E = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t a = where[i];
        float *pa = cl.cpos + 3 * a;
        int32_t n = cl.n;
        float inv_cell = (float)((double)n / (double)L);
        int64_t c = cell_coord(pa[0], inv_cell, n) +
                    (int64_t)n * (cell_coord(pa[1], inv_cell, n) + (int64_t)n * cell_coord(pa[2], inv_cell, n));
        int64_t nbc[27];
        int nnb = neighbour_cells(&cl, c, nbc), nb = 0;
        for (int s = 0; s < nnb; ++s)
            for (int64_t k = cl.start[nbc[s]]; k < cl.start[nbc[s] + 1]; ++k) {
                int32_t j = cl.idx[k];
                if (j > i && orc_dist2(pa, cl.cpos + 3 * k, L) < rc2)
                    buf[nb++] = j;
            }
        qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
        for (int s = 0; s < nb; ++s) {
            if (E < cap) {
                int32_t j = buf[s];
                float d2 = orc_dist2(pos + 3 * i, pos + 3 * j, L);
                float d = sqrtf(d2);
                pi[E] = (int32_t)i;
                pj[E] = j;
                pd[E] = d;
                pp[E] = orc_edge_prob(d, d2, b, b2, form, coef);
            }
            ++E;
        }
    }
    free(where); free(buf); cell_list_free(&cl);
    return E;
}

/* Per-sample FoF over the sampled edges (Sec. 3.2, Eq. 8): edge e is present
   in sample k iff u(seed, i_e, j_e, k) < p_e.  labels: [K,N] smallest index
   per component; n_halos[k] = number of components with >= min_size members. */
int orc_reinforce_sample(int64_t N, int64_t E, const int32_t *pi, const int32_t *pj,
                         const float *pp, int32_t K, uint64_t seed, int32_t min_size,
                         int32_t *labels, int32_t *n_halos)
{
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * N);
    if (!cnt)
        return ORC_ENOMEM;
    for (int32_t k = 0; k < K; ++k) {
        int32_t *lab = labels + (int64_t)k * N;
        for (int64_t i = 0; i < N; ++i)
            lab[i] = (int32_t)i;
        for (int64_t e = 0; e < E; ++e)
            if (orc_edge_uniform(seed, pi[e], pj[e], k) < pp[e])
                uf_union(lab, pi[e], pj[e]);
        for (int64_t i = 0; i < N; ++i) {
            lab[i] = uf_find(lab, (int32_t)i);
            cnt[i] = 0;
        }
        for (int64_t i = 0; i < N; ++i)
            cnt[lab[i]] += 1;
        int32_t h = 0;
        for (int64_t i = 0; i < N; ++i)
            if (lab[i] == i && cnt[i] >= min_size)
                ++h;
        n_halos[k] = h;
    }
    free(cnt);
    return ORC_OK;
}

/* Score-function gradient (Eqs. 6-7) with respect to positions, FP64:
     log p(y) = sum_e [y_e log p_e + (1-y_e) log(1-p_e)],
     d log p(y) / d z_e = y_e - p_e,
     form 0: z_e = (b - d_e)/tau     -> dz/dx_i = (x_j - x_i)_mi / (tau d_e)
     form 1: z_e = alpha (b2-d2)/b2  -> dz/dx_i = 2 (alpha/b2) (x_j - x_i)_mi
   and dz/dx_j = -dz/dx_i.  g = (1/K) sum_k A_k d log p(y_k) / dx.
   coef is 1/tau (form 0) or alpha/b2 (form 1).  d_e = 0 contributes 0. */
int orc_reinforce_grad(const float *pos, int64_t N, float L, int64_t E,
                       const int32_t *pi, const int32_t *pj, const float *pp,
                       int32_t K, uint64_t seed, const double *adv, int32_t form,
                       double coef, double *g)
{
    for (int64_t i = 0; i < 3 * N; ++i)
        g[i] = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        int32_t i = pi[e], j = pj[e];
        double s = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            double y = orc_edge_uniform(seed, i, j, k) < pp[e] ? 1.0 : 0.0;
            s += adv[k] * (y - (double)pp[e]);
        }
        s /= (double)K;
        double dx[3], d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            dx[a] = mi_f64((double)pos[3 * j + a] - (double)pos[3 * i + a], (double)L);
            d2 += dx[a] * dx[a];
        }
        double fac;
        if (form == 0) {
            double d = sqrt(d2);
            fac = d > 0.0 ? coef / d : 0.0;
        } else {
            fac = 2.0 * coef;
        }
        for (int a = 0; a < 3; ++a) {
            g[3 * i + a] += s * fac * dx[a];
            g[3 * j + a] -= s * fac * dx[a];
        }
    }
    (void)N;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Helpers for checks at full size: the same definitions, restricted.        */

/* Sample k alone (labels [N], smallest member index; *n_halos). */
int orc_reinforce_sample_one(int64_t N, int64_t E, const int32_t *pi, const int32_t *pj,
                             const float *pp, int32_t k, uint64_t seed, int32_t min_size,
                             int32_t *lab, int32_t *n_halos)
{
    int64_t *cnt = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    if (!cnt)
        return ORC_ENOMEM;
    for (int64_t i = 0; i < N; ++i)
        lab[i] = (int32_t)i;
    for (int64_t e = 0; e < E; ++e)
        if (orc_edge_uniform(seed, pi[e], pj[e], k) < pp[e])
            uf_union(lab, pi[e], pj[e]);
    for (int64_t i = 0; i < N; ++i)
        lab[i] = uf_find(lab, (int32_t)i);
    for (int64_t i = 0; i < N; ++i)
        cnt[lab[i]] += 1;
    int32_t h = 0;
    for (int64_t i = 0; i < N; ++i)
        if (lab[i] == i && cnt[i] >= min_size)
            ++h;
    *n_halos = h;
    free(cnt);
    return ORC_OK;
}

/* The score-function gradient of orc_reinforce_grad, evaluated only for the
   particles with mask[i] != 0 (other rows are left 0). */
int orc_reinforce_grad_masked(const float *pos, int64_t N, float L, int64_t E,
                              const int32_t *pi, const int32_t *pj, const float *pp,
                              int32_t K, uint64_t seed, const double *adv, int32_t form,
                              double coef, const uint8_t *mask, double *g)
{
    for (int64_t i = 0; i < 3 * N; ++i)
        g[i] = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        int32_t i = pi[e], j = pj[e];
        if (!mask[i] && !mask[j])
            continue;
        double s = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            double y = orc_edge_uniform(seed, i, j, k) < pp[e] ? 1.0 : 0.0;
            s += adv[k] * (y - (double)pp[e]);
        }
        s /= (double)K;
        double dx[3], d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            dx[a] = mi_f64((double)pos[3 * j + a] - (double)pos[3 * i + a], (double)L);
            d2 += dx[a] * dx[a];
        }
        double fac = form == 0 ? (d2 > 0.0 ? coef / sqrt(d2) : 0.0) : 2.0 * coef;
        for (int a = 0; a < 3; ++a) {
            if (mask[i])
                g[3 * i + a] += s * fac * dx[a];
            if (mask[j])
                g[3 * j + a] -= s * fac * dx[a];
        }
    }
    return ORC_OK;
}

/* Element-wise orc_exp over an array. */
void orc_exp_array(const float *x, float *y, int64_t n)
{
    for (int64_t t = 0; t < n; ++t)
        y[t] = orc_exp(x[t]);
}
