// api_stream.cu -- FoF over slabs of cell layers: the box is cut into n_slabs
// slabs of whole z-layers of the cell grid; each slab's particles, with one
// extra cell layer on each side (periodic), are linked on the GPU with the
// ordinary bin + link path, and the slabs' components are fused by a
// union-find over global particle indices.  This is the streaming mode of
// Sec. 2.2 (memory bounded by the largest slab instead of the whole box) and
// the slab decomposition with union-find fusion of Sec. 2.3 (the same merge
// serves several devices, each holding one slab).
//
// Why it is exact: cells are at least 1.01 b wide, so every friend of a
// particle lies in its own or an adjacent cell; the particles of a slab's
// layers plus one layer on each side therefore contain every friend of the
// slab's own ("core") particles.  Linking that subset in the full periodic
// box finds only true links, and every true link has a core end in some slab,
// so the union of the slabs' links is the friendship graph.  Slab s's
// components are connected subgraphs; particles of the extra layers belong to
// two slabs and join their components.  The subset is listed in ascending
// global index, so a slab's raw label (smallest subset index) maps to the
// smallest global index of that slab component, and the fused root (smaller
// index wins) is the smallest global index of the true component.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "jfof_internal.cuh"
#include "k_fof.cuh"

using namespace jfof;

namespace {

// Host threads for the host-side passes.
int host_threads() {
    unsigned t = std::thread::hardware_concurrency();
    if (t < 1) t = 1;
    if (t > 64) t = 64;
    return int(t);
}

// f(t, lo, hi) over T contiguous chunks of [0, n).
template <class F>
void par_chunks(int64_t n, int T, F f) {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) {
        int64_t lo = n * t / T, hi = n * (t + 1) / T;
        th.emplace_back([=] { f(t, lo, hi); });
    }
    for (auto &x : th) x.join();
}

// z cell layer of a position: the device's cell coordinate (one binary32
// multiply by f32(n/L), floor, clamp to [0, n-1]).
inline int z_layer(float z, float inv_cell, int n) {
    float u = z * inv_cell;
    int c = int(std::floor(u));
    return c < 0 ? 0 : (c > n - 1 ? n - 1 : c);
}

struct SlabGeom {
    int n, S;
    float inv_cell;
    // layers of slab s: [z0, z1); the subset adds z0 - 1 and z1 (mod n)
    int z0(int s) const { return int(int64_t(n) * s / S); }
    int z1(int s) const { return int(int64_t(n) * (s + 1) / S); }
    bool in_subset(int c, int s) const {
        int span = z1(s) - z0(s) + 2;
        if (span >= n) return true;
        int d = c - (z0(s) - 1);
        d = ((d % n) + n) % n;
        return d < span;
    }
    bool is_core(int c, int s) const { return c >= z0(s) && c < z1(s); }
};

int check_stream_args(const float *h_pos, int64_t N, float L, float b, int32_t n_axis, int32_t n_slabs, int *n_out) {
    if (!h_pos) return JFOF_EINVAL;
    int e = check_box(N, L, b);
    if (e) return e;
    int32_t n;
    if ((e = resolve_n(N, L, b, n_axis, &n))) return e;
    if (n < 3 || n_slabs < 1 || n_slabs > n) return JFOF_EINVAL;
    *n_out = n;
    return JFOF_OK;
}

// Every coordinate finite and inside [0, L).
bool positions_in_box(const float *h_pos, int64_t N, float L) {
    const int T = host_threads();
    std::vector<char> ok(T, 1);
    par_chunks(3 * N, T, [&](int t, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            if (!(h_pos[i] >= 0.0f && h_pos[i] < L)) {
                ok[t] = 0;
                return;
            }
    });
    return std::all_of(ok.begin(), ok.end(), [](char c) { return c != 0; });
}

// z layer of every particle.
std::vector<int32_t> layers_of(const float *h_pos, int64_t N, const SlabGeom &sg) {
    std::vector<int32_t> lay(static_cast<size_t>(N));
    par_chunks(N, host_threads(), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) lay[size_t(i)] = z_layer(h_pos[3 * i + 2], sg.inv_cell, sg.n);
    });
    return lay;
}

// Ascending global indices of slab s's subset (and, if core is given, 1 for
// its core particles).  Returns the subset size.
int64_t select_subset(const std::vector<int32_t> &lay, const SlabGeom &sg, int s, int64_t *idx, uint8_t *core) {
    const int64_t N = int64_t(lay.size());
    const int T = host_threads();
    std::vector<int64_t> cnt(T + 1, 0);
    par_chunks(N, T, [&](int t, int64_t lo, int64_t hi) {
        int64_t c = 0;
        for (int64_t i = lo; i < hi; ++i) c += sg.in_subset(lay[size_t(i)], s);
        cnt[t + 1] = c;
    });
    for (int t = 0; t < T; ++t) cnt[t + 1] += cnt[t];
    if (idx || core)
        par_chunks(N, T, [&](int t, int64_t lo, int64_t hi) {
            int64_t w = cnt[t];
            for (int64_t i = lo; i < hi; ++i) {
                const int c = lay[size_t(i)];
                if (!sg.in_subset(c, s)) continue;
                if (idx) idx[w] = i;
                if (core) core[w] = sg.is_core(c, s) ? 1 : 0;
                ++w;
            }
        });
    return cnt[T];
}

int32_t uf_root(std::vector<int32_t> &par, int32_t x) {
    int32_t r = x;
    while (par[size_t(r)] != r) r = par[size_t(r)];
    while (par[size_t(x)] != r) {
        int32_t nx = par[size_t(x)];
        par[size_t(x)] = r;
        x = nx;
    }
    return r;
}

void uf_join(std::vector<int32_t> &par, int32_t a, int32_t b) {
    a = uf_root(par, a);
    b = uf_root(par, b);
    if (a == b) return;
    if (a < b) par[size_t(b)] = a;
    else par[size_t(a)] = b;
}

// Device bytes of one slab: positions, labels and the bin/link workspace.
size_t slab_bytes(int64_t Ns, int n) {
    return align_up(sizeof(float) * 3 * size_t(Ns)) + align_up(sizeof(int32_t) * size_t(Ns)) + fof_layout(Ns, n, nullptr, nullptr);
}

}  // namespace

extern "C" {

int jfof_slab_select(const float *h_pos, int64_t N, float L, float b, int32_t n_axis, int32_t n_slabs,
                     int32_t slab, int64_t *h_idx, uint8_t *h_core, int64_t *n_sel) {
    int n;
    int e = check_stream_args(h_pos, N, L, b, n_axis, n_slabs, &n);
    if (e) return e;
    if (!n_sel || slab < 0 || slab >= n_slabs) return JFOF_EINVAL;
    if (!positions_in_box(h_pos, N, L)) return JFOF_ERANGE;
    SlabGeom sg{n, n_slabs, float(double(n) / double(L))};
    std::vector<int32_t> lay = layers_of(h_pos, N, sg);
    *n_sel = select_subset(lay, sg, slab, h_idx, h_core);
    return JFOF_OK;
}

int jfof_merge_labels(int64_t N, const int32_t *h_pre, int64_t n_pairs, const int32_t *h_a, const int32_t *h_b,
                      int32_t *h_label) {
    if (N < 1 || N > int64_t(INT32_MAX) || !h_pre || !h_label || n_pairs < 0 || (n_pairs > 0 && (!h_a || !h_b)))
        return JFOF_EINVAL;
    for (int64_t k = 0; k < n_pairs; ++k)
        if (h_a[k] < 0 || h_a[k] >= N || h_b[k] < 0 || h_b[k] >= N) return JFOF_EINVAL;
    std::vector<int32_t> par(static_cast<size_t>(N));
    for (int64_t i = 0; i < N; ++i) {
        if (h_pre[i] < 0 || h_pre[i] >= N) return JFOF_EINVAL;
        par[size_t(i)] = int32_t(i);
    }
    for (int64_t k = 0; k < n_pairs; ++k) uf_join(par, h_a[k], h_b[k]);
    for (int64_t i = 0; i < N; ++i) h_label[i] = uf_root(par, h_pre[i]);
    return JFOF_OK;
}

int jfof_fof_stream_bytes(const float *h_pos, int64_t N, float L, float b, int32_t n_axis, int32_t n_slabs,
                          size_t *bytes) {
    int n;
    int e = check_stream_args(h_pos, N, L, b, n_axis, n_slabs, &n);
    if (e) return e;
    if (!bytes) return JFOF_EINVAL;
    if (!positions_in_box(h_pos, N, L)) return JFOF_ERANGE;
    SlabGeom sg{n, n_slabs, float(double(n) / double(L))};
    std::vector<int32_t> lay = layers_of(h_pos, N, sg);
    int64_t mx = 1;
    for (int s = 0; s < n_slabs; ++s) mx = std::max(mx, select_subset(lay, sg, s, nullptr, nullptr));
    *bytes = slab_bytes(mx, n);
    return JFOF_OK;
}

int jfof_fof_stream(jfof_ctx *ctx, const float *h_pos, int64_t N, float L, float b, int32_t n_axis,
                    int32_t n_slabs, int32_t min_size, void *ws, size_t ws_bytes, int32_t *h_label,
                    int32_t *h_halo_id, int64_t *n_halos) {
    if (!ctx || !ws || !h_label || min_size < 1) return JFOF_EINVAL;
    int n;
    int e = check_stream_args(h_pos, N, L, b, n_axis, n_slabs, &n);
    if (e) return e;
    if (!positions_in_box(h_pos, N, L)) return JFOF_ERANGE;
    SlabGeom sg{n, n_slabs, float(double(n) / double(L))};
    std::vector<int32_t> lay = layers_of(h_pos, N, sg);
    std::vector<int64_t> sizes(static_cast<size_t>(n_slabs));
    int64_t mx = 1;
    for (int s = 0; s < n_slabs; ++s) {
        sizes[size_t(s)] = select_subset(lay, sg, s, nullptr, nullptr);
        mx = std::max(mx, sizes[size_t(s)]);
    }
    if (ws_bytes < slab_bytes(mx, n)) return JFOF_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return JFOF_ECUDA;
    CtxScope scope(ctx);
    char *base = reinterpret_cast<char *>(ws);
    float *d_pos = reinterpret_cast<float *>(base);
    int32_t *d_lab = reinterpret_cast<int32_t *>(base + align_up(sizeof(float) * 3 * size_t(mx)));
    void *d_ws = base + align_up(sizeof(float) * 3 * size_t(mx)) + align_up(sizeof(int32_t) * size_t(mx));

    // pre[g]: the label of particle g in its own slab; pairs: the labels a
    // particle of an extra layer has in its own slab and in the neighbour's
    std::vector<int32_t> pre(static_cast<size_t>(N), -1);
    std::vector<int32_t> ga, gr;  // ghost records (global index, label in this slab)
    std::vector<int64_t> idx(static_cast<size_t>(mx));
    std::vector<uint8_t> core(static_cast<size_t>(mx));
    std::vector<float> hp(3 * static_cast<size_t>(mx));
    std::vector<int32_t> lab(static_cast<size_t>(mx));
    const int T = host_threads();
    for (int s = 0; s < n_slabs; ++s) {
        const int64_t Ns = sizes[size_t(s)];
        if (Ns == 0) continue;
        select_subset(lay, sg, s, idx.data(), core.data());
        par_chunks(Ns, T, [&](int, int64_t lo, int64_t hi) {
            for (int64_t j = lo; j < hi; ++j) std::memcpy(&hp[3 * size_t(j)], h_pos + 3 * idx[size_t(j)], 12);
        });
        if (cudaMemcpyAsync(d_pos, hp.data(), sizeof(float) * 3 * size_t(Ns), cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess)
            return JFOF_ECUDA;
        FofBuffers fb;
        fof_layout(Ns, n, &fb, d_ws);
        LinkParams lp = make_link_params(Ns, L, b, n, ctx->small_threshold, ctx->dense_threshold, ctx->cta_shape);
        launch_bin_cells(d_pos, Ns, L, n, false, lp, fb, ctx->dev(), ctx->stream);
        jfof_cells c{};
        c.n = Ns;
        c.n_axis = n;
        c.brick = kBrick;
        c.L = L;
        c.b = b;
        c.small_threshold = lp.S;
        c.dense_threshold = lp.T;
        c.spos = fb.spos;
        c.cell_start = fb.cell_start;
        c.n_cells_table = cell_table_entries(n);
        c.workspace = d_ws;
        launch_link(c, fb, lp, d_lab, ctx->dev(), ctx->stream);
        if (cudaGetLastError() != cudaSuccess) return JFOF_ECUDA;
        if (cudaMemcpyAsync(lab.data(), d_lab, sizeof(int32_t) * size_t(Ns), cudaMemcpyDeviceToHost, ctx->stream) !=
            cudaSuccess)
            return JFOF_ECUDA;
        if ((e = jfof_sync(ctx))) return e;
        for (int64_t j = 0; j < Ns; ++j) {
            const int32_t g = int32_t(idx[size_t(j)]);
            const int32_t r = int32_t(idx[size_t(lab[size_t(j)])]);
            if (core[size_t(j)]) {
                pre[size_t(g)] = r;
            } else {
                ga.push_back(g);
                gr.push_back(r);
            }
        }
    }
    // fuse: a particle of an extra layer joins its label here with its label
    // in its own slab
    std::vector<int32_t> a(ga.size());
    for (size_t k = 0; k < ga.size(); ++k) a[k] = pre[size_t(ga[k])];
    if ((e = jfof_merge_labels(N, pre.data(), int64_t(a.size()), a.data(), gr.data(), h_label))) return e;
    // groups: count per raw label, the cut, halo ids ascending by raw label
    if (h_halo_id || n_halos) {
        std::vector<int32_t> cnt(static_cast<size_t>(N), 0);
        for (int64_t i = 0; i < N; ++i) ++cnt[size_t(h_label[i])];
        int64_t H = 0;
        for (int64_t r = 0; r < N; ++r) cnt[size_t(r)] = (h_label[r] == r && cnt[size_t(r)] >= min_size) ? int32_t(H++) : -1;
        if (h_halo_id)
            for (int64_t i = 0; i < N; ++i) h_halo_id[i] = cnt[size_t(h_label[i])];
        if (n_halos) *n_halos = H;
    }
    return JFOF_OK;
}

}  // extern "C"
