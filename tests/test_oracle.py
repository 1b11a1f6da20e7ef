"""Pins for the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test names the passage it follows.

A plausible mistake in the oracle -- a dropped link (grid too coarse/fine, a
missed wrap), a wrong comparison (< vs <=), a wrong normalisation (n vs n-1),
a sign error in a gradient -- fails at least one of these.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def partition(labels):
    """Canonical partition: frozenset of frozensets of indices."""
    groups = {}
    for i, l in enumerate(labels):
        groups.setdefault(int(l), []).append(i)
    return frozenset(frozenset(v) for v in groups.values())


# --------------------------------------------------------------------------
# Labels (Sec. 1, Sec. 2 steps (iii)-(v), Algorithm 2)

def test_hand_cases_golden():
    cases = json.load(open(os.path.join(GOLDEN, "fof_hand_cases.json")))["cases"]
    for c in cases:
        pos = np.array(c["pos"], np.float32)
        got = oracle.fof_labels(pos, c["L"], c["b"])
        assert got.tolist() == c["labels"], c["name"]
        assert oracle.fof_brute(pos, c["L"], c["b"]).tolist() == c["labels"], c["name"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cell_list_equals_brute_force_uniform(seed):
    # dense uniform box with b near the percolation scale: many mixed groups
    N, L = 3000, 10.0
    pos = synth.uniform(N, L, seed).numpy()
    b = 0.55 * L / N ** (1 / 3)
    bf = oracle.fof_brute(pos, L, b)
    for n in (0, 1, 3, 4, oracle.max_cells_per_axis(L, b)):
        assert np.array_equal(oracle.fof_labels(pos, L, b, n_axis=n), bf), n


def test_cell_list_equals_brute_force_clustered():
    spec = synth.BoxSpec("t", 4096, 40.0, synth.linking_length(40.0, 4096) * 2.0, 40, 0.5, 3)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    bf = oracle.fof_brute(pos, spec.L, spec.b)
    assert np.array_equal(oracle.fof_labels(pos, spec.L, spec.b), bf)
    assert len(set(bf.tolist())) < 4096 - 100  # the clustered box really has groups


def test_cell_list_equals_brute_force_near_boundary():
    # particles hugging the six faces: every link crosses the periodic boundary
    rng = np.random.default_rng(5)
    N, L, b = 2000, 8.0, 0.3
    p = rng.uniform(0, L, (N, 3))
    face = rng.integers(0, 3, N)
    side = rng.integers(0, 2, N)
    p[np.arange(N), face] = np.where(side == 0, rng.uniform(0, 0.2, N), L - rng.uniform(1e-6, 0.2, N))
    p = p.astype(np.float32)
    p[p >= L] = 0
    bf = oracle.fof_brute(p, L, b)
    assert np.array_equal(oracle.fof_labels(p, L, b), bf)
    # some group spans the boundary
    spans = False
    for g in partition(bf):
        idx = list(g)
        if len(idx) > 1:
            xs = p[idx]
            if (xs.max(0) - xs.min(0)).max() > L / 2:
                spans = True
                break
    assert spans


# The threaded oracle (slabs of cell layers, Sec. 2.3's union-find fusion with
# threads for devices) must give the sequential oracle's labels, which the
# brute-force pins above fix, for any thread count and grid -- including more
# threads than layers (empty slabs) and one-layer slabs whose every pair
# crosses into a neighbour slab.

@pytest.mark.parametrize("threads", [1, 2, 3, 5, 8])
def test_threaded_labels_equal_sequential_uniform(threads):
    N, L = 3000, 10.0
    pos = synth.uniform(N, L, 0).numpy()
    b = 0.55 * L / N ** (1 / 3)
    bf = oracle.fof_brute(pos, L, b)
    for n in (0, 1, 3, 4, 7, oracle.max_cells_per_axis(L, b)):
        assert np.array_equal(oracle.fof_labels_mt(pos, L, b, n_axis=n, threads=threads), bf), (n, threads)


def test_threaded_labels_equal_sequential_clustered_and_boundary():
    spec = synth.BoxSpec("t", 20000, 40.0, synth.linking_length(40.0, 20000) * 1.5, 120, 0.6, 4)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    seq = oracle.fof_labels(pos, spec.L, spec.b)
    assert len(set(seq.tolist())) < 20000 - 1000
    for t in (2, 4, 7, 16):
        assert np.array_equal(oracle.fof_labels_mt(pos, spec.L, spec.b, threads=t), seq), t
    # particles hugging the periodic faces: slab 0 and the last slab link
    rng = np.random.default_rng(6)
    L, b = 10.0, 0.4
    q = rng.uniform(0, L, (4000, 3))
    q[:, 2] = np.where(rng.random(4000) < 0.5, rng.uniform(0, 0.3, 4000), rng.uniform(L - 0.3, L, 4000))
    q = q.astype(np.float32)
    bf = oracle.fof_brute(q, L, b)
    assert any(bf[i] != i for i in range(4000))
    for t in (2, 3, 6):
        assert np.array_equal(oracle.fof_labels_mt(q, L, b, threads=t), bf), t


@pytest.mark.parametrize("m", [4, 7])
def test_cubic_lattice_closed_form(m):
    # lattice spacing a: a = 0.9 b -> one periodic group; a = 1.1 b -> singletons
    a = 1.0
    idx = np.arange(m, dtype=np.float32)
    gz, gy, gx = np.meshgrid(idx, idx, idx, indexing="ij")
    pos = np.stack([gx, gy, gz], -1).reshape(-1, 3).astype(np.float32) * np.float32(a)
    L = m * a
    one = oracle.fof_labels(pos, L, a / 0.9)
    assert (one == 0).all()
    single = oracle.fof_labels(pos, L, a / 1.1)
    assert np.array_equal(single, np.arange(m ** 3))


def test_chain_across_boundary_links_end_to_end():
    L, b = 20.0, 0.5
    s = np.float32(0.99 * b)
    xs = (np.float32(L) - np.float32(3.0) + s * np.arange(14, dtype=np.float32)) % np.float32(L)
    pos = np.stack([xs, np.full_like(xs, 5.0), np.full_like(xs, 5.0)], -1).astype(np.float32)
    perm = np.random.default_rng(1).permutation(len(xs))
    lab = oracle.fof_labels(pos[perm], L, b)
    assert len(set(lab.tolist())) == 1 and lab[0] == 0
    # second chain 1.01 b away along y: two groups
    pos2 = pos.copy()
    pos2[:, 1] += np.float32(1.01 * b)
    both = np.concatenate([pos, pos2]).astype(np.float32)
    lab2 = oracle.fof_labels(both, L, b)
    assert len(set(lab2.tolist())) == 2


def test_invariants_on_clustered_box():
    spec = synth.BoxSpec("t", 6000, 50.0, synth.linking_length(50.0, 6000) * 1.5, 60, 0.5, 7)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    L, b = spec.L, spec.b
    lab = oracle.fof_labels(pos, L, b)
    b2 = np.float32(b) * np.float32(b)
    # label = smallest member, label of label is itself
    for g in partition(lab):
        assert lab[min(g)] == min(g) and all(lab[i] == min(g) for i in g)
    # no linked pair spans two groups (vectorised float32 predicate)
    hL = np.float32(0.5 * L)
    for i in range(0, len(pos), 500):
        blk = pos[i:i + 500]
        d = pos[None, :, :] - blk[:, None, :]
        d = np.where(d > hL, d - np.float32(L), np.where(d < -hL, d + np.float32(L), d)).astype(np.float32)
        sq = d * d
        d2 = (sq[..., 0] + sq[..., 1]) + sq[..., 2]
        ii, jj = np.nonzero(d2 <= b2)
        assert np.array_equal(lab[i + ii], lab[jj])
    # each group is connected (BFS over the predicate inside the group)
    for g in partition(lab):
        if len(g) < 2:
            continue
        idx = sorted(g)
        sub = pos[idx]
        d = sub[None] - sub[:, None]
        d = np.where(d > hL, d - np.float32(L), np.where(d < -hL, d + np.float32(L), d)).astype(np.float32)
        sq = d * d
        adj = ((sq[..., 0] + sq[..., 1]) + sq[..., 2]) <= b2
        seen = {0}
        frontier = [0]
        while frontier:
            k = frontier.pop()
            for j in np.nonzero(adj[k])[0]:
                if j not in seen:
                    seen.add(int(j))
                    frontier.append(int(j))
        assert len(seen) == len(idx)


def test_labels_invariant_under_permutation_and_grid():
    spec = synth.BoxSpec("t", 5000, 30.0, synth.linking_length(30.0, 5000) * 1.6, 30, 0.5, 11)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    base = partition(oracle.fof_labels(pos, spec.L, spec.b))
    perm = np.random.default_rng(3).permutation(len(pos))
    lab_p = oracle.fof_labels(pos[perm], spec.L, spec.b)
    mapped = frozenset(frozenset(int(perm[i]) for i in g) for g in partition(lab_p))
    assert mapped == base
    for n in (3, 5, oracle.max_cells_per_axis(spec.L, spec.b)):
        assert partition(oracle.fof_labels(pos, spec.L, spec.b, n_axis=n)) == base


def test_strict_vs_nonstrict_tie():
    L, b = 16.0, 0.375  # 0.375 exact; 1.0 + 0.375 exact
    pos = np.array([[1.0, 2.0, 2.0], [1.375, 2.0, 2.0]], np.float32)
    assert oracle.fof_labels(pos, L, b).tolist() == [0, 0]
    nb = np.nextafter(np.float32(b), np.float32(0))
    assert oracle.fof_labels(pos, L, float(nb)).tolist() == [0, 1]


def test_wrap_reading():
    L = 10.0
    p = np.array([[-0.5, 10.0, 25.0], [9.999999, -1e-9, 3.0]], np.float32)
    w = oracle.wrap(p, L)
    assert (w >= 0).all() and (w < L).all()
    assert np.isclose(w[0, 0], 9.5) and w[0, 1] == 0.0 and np.isclose(w[0, 2], 5.0)
    assert w[1, 2] == np.float32(3.0)


def test_rejects_out_of_range_and_bad_b():
    pos = np.array([[0.1, 0.2, 10.0]], np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.fof_labels(pos, 10.0, 0.2)
    with pytest.raises(oracle.OracleError):
        oracle.fof_labels(np.zeros((1, 3), np.float32), 10.0, 5.0)


# --------------------------------------------------------------------------
# Groups (Sec. 2 step (vi))

def test_groups_cut_19_20_21():
    sizes = [19, 20, 21, 1, 40]
    lab = []
    base = 0
    roots = []
    for s in sizes:
        roots.append(base)
        lab += [base] * s
        base += s
    lab = np.array(lab, np.int32)
    hid, cnt = oracle.groups(lab, 20)
    assert cnt.tolist() == [20, 21, 40]
    assert (hid[:19] == -1).all()
    assert (hid[19:39] == 0).all() and (hid[39:60] == 1).all()
    assert hid[60] == -1 and (hid[61:] == 2).all()


def test_groups_conservation_and_order():
    spec = synth.BoxSpec("t", 8000, 30.0, synth.linking_length(30.0, 8000), 50, 0.6, 2)
    pos, _ = synth.generate(spec, velocities=False)
    lab = oracle.fof_labels(pos.numpy(), spec.L, spec.b)
    hid, cnt = oracle.groups(lab, 5)
    assert cnt.sum() + (hid < 0).sum() == len(lab)
    H = len(cnt)
    assert set(hid[hid >= 0].tolist()) == set(range(H))
    firsts = [np.nonzero(hid == h)[0].min() for h in range(H)]
    assert firsts == sorted(firsts)
    for h in range(H):
        assert (hid == h).sum() == cnt[h]


# --------------------------------------------------------------------------
# Properties (Sec. 3.1, Eq. 4; Table 1) and their adjoint

def test_props_closed_forms():
    L = 10.0
    c = np.array([0.0, 9.99, 5.0])
    offs = np.array(list(itertools.product([-0.1, 0.1], repeat=3)))
    pos = ((c + offs) % L).astype(np.float32)
    s = 7.0
    vel = (np.array([20.0, -3.0, 1.0]) + s * np.sign(offs)).astype(np.float32)
    hid = np.zeros(8, np.int32)
    mass, com, vmean, sigv = oracle.halo_props(pos, vel, hid, 1, L, particle_mass=2.5)
    assert mass[0] == 20.0
    err = np.abs(((com[0] - c) + L / 2) % L - L / 2)
    assert err.max() < 1e-6
    assert np.allclose(vmean[0], [20.0, -3.0, 1.0])
    assert abs(sigv[0] - s) < 1e-12
    vel2 = np.tile(np.array([[3.0, 4.0, 5.0]], np.float32), (8, 1))
    _, _, _, sg = oracle.halo_props(pos, vel2, hid, 1, L)
    assert sg[0] == 0.0


def _cold_halo_with_outlier(n=2400, L=100.0, seed=21):
    """A cold, fast halo whose smallest-index member is a velocity outlier and
    sits at the halo's edge (positions and velocities in binary32)."""
    rng = np.random.default_rng(seed)
    c = np.array([L - 0.05, 0.02, 50.0])  # straddles two periodic faces
    pos = (c + rng.normal(0.0, 0.03, (n, 3))) % L
    pos[0] = (c + np.array([0.25, -0.2, 0.22])) % L
    v0 = np.array([812.0, -640.0, 377.0])
    vel = v0 + rng.normal(0.0, 0.05, (n, 3))
    vel[0] = v0 + np.array([900.0, -750.0, 820.0])  # outlier, ~2e4 sigma away
    return pos.astype(np.float32), vel.astype(np.float32), L


def test_props_cold_halo_with_outlier_first_member():
    # velocity dispersion (population, 1-D) of a cold halo whose reference
    # member is an outlier: FP64 two-pass oracle == numpy's variance of the
    # 3n deviations (a library routine), and the periodic COM == the plain
    # mean of the unwrapped positions
    pos, vel, L = _cold_halo_with_outlier()
    n = pos.shape[0]
    hid = np.zeros(n, np.int32)
    m, com, vm, sg = oracle.halo_props(pos.astype(np.float64), vel.astype(np.float64), hid, 1, L)
    v64 = vel.astype(np.float64)
    assert np.allclose(vm[0], v64.mean(0), rtol=0, atol=1e-12)
    want = math.sqrt(np.var(v64 - v64.mean(0), axis=0, ddof=0).sum() / 3.0)
    assert abs(sg[0] - want) <= 1e-12 * want
    unwrapped = pos.astype(np.float64).copy()
    ref0 = unwrapped[0].copy()
    unwrapped = ref0 + (unwrapped - ref0 + L / 2) % L - L / 2
    assert np.allclose(com[0], unwrapped.mean(0) % L, rtol=0, atol=1e-9)
    # the outlier dominates the one-pass sums shifted by it: |vbar - v_r|^2 /
    # sigma^2 is about 3n, so such a sum would lose about 3n ulp of sigma^2
    assert np.sum((vm[0] - v64[0]) ** 2) / sg[0] ** 2 > 2 * n


def test_props_unassigned_ignored_and_two_halos():
    pos = np.array([[1, 1, 1], [1.2, 1, 1], [5, 5, 5], [9.9, 0, 0], [0.1, 0, 0]], np.float32)
    vel = np.array([[1, 0, 0], [3, 0, 0], [100, 100, 100], [0, 2, 0], [0, 4, 0]], np.float32)
    hid = np.array([0, 0, -1, 1, 1], np.int32)
    m, com, vm, sg = oracle.halo_props(pos, vel, hid, 2, 10.0)
    assert np.allclose(com[0], [1.1, 1, 1])
    # the pair at x = 9.9 and 0.1 straddles the boundary: COM at x = 0 (mod L)
    assert min(abs(com[1][0]), abs(com[1][0] - 10.0)) < 1e-6 and 0 <= com[1][0] < 10.0
    assert np.allclose(vm[0], [2, 0, 0]) and np.allclose(vm[1], [0, 3, 0])
    assert np.isclose(sg[0], math.sqrt(2.0 / 6.0)) and np.isclose(sg[1], math.sqrt(2.0 / 6.0))


def _loss_and_props(pos64, vel64, hid, H, L, w):
    m, com, vm, sg = oracle.halo_props(pos64, vel64, hid, H, L)
    return float(np.sum(w * (np.sum(com ** 2, 1) + sg ** 2))), com, vm, sg


def test_backward_matches_central_differences():
    # loss = sum_h w_h (|com_h|^2 + sigma_h^2) with frozen memberships
    spec = synth.BoxSpec("t", 3000, 20.0, synth.linking_length(20.0, 3000) * 1.5, 25, 0.6, 4)
    pos, vel = synth.generate(spec)
    pos64, vel64 = pos.numpy().astype(np.float64), vel.numpy().astype(np.float64)
    lab = oracle.fof_labels(pos.numpy(), spec.L, spec.b)
    hid, cnt = oracle.groups(lab, 5)
    H = len(cnt)
    assert H > 3
    w = np.random.default_rng(0).uniform(0, 1, H)
    f0, com, vm, sg = _loss_and_props(pos64, vel64, hid, H, spec.L, w)
    gp, gv = oracle.halo_props_backward(vel64, hid, H, vm, sg,
                                        g_com=2 * w[:, None] * com, g_sigv=2 * w * sg)
    rng = np.random.default_rng(1)
    members = np.nonzero(hid >= 0)[0]
    eps = 1e-6 * spec.L
    for i in rng.choice(members, 12, replace=False):
        for a in range(3):
            for arr, g in ((pos64, gp), (vel64, gv)):
                e = eps if arr is pos64 else 1e-4
                arr[i, a] += e
                fp = _loss_and_props(pos64, vel64, hid, H, spec.L, w)[0]
                arr[i, a] -= 2 * e
                fm = _loss_and_props(pos64, vel64, hid, H, spec.L, w)[0]
                arr[i, a] += e
                fd = (fp - fm) / (2 * e)
                assert abs(fd - g[i, a]) <= 1e-5 * max(1.0, abs(fd)), (i, a, fd, g[i, a])
    nonmem = np.nonzero(hid < 0)[0]
    assert (gp[nonmem] == 0).all() and (gv[nonmem] == 0).all()


def test_backward_analytic_closed_form():
    # C5a closed form: g_x_i = 2 w_h com_h / n_h ; g_v_i = 2 w_h (v_i - vbar_h) / (3 n_h)
    rng = np.random.default_rng(2)
    n = 9
    pos = rng.uniform(3, 4, (n, 3))
    vel = rng.normal(0, 5, (n, 3))
    hid = np.zeros(n, np.int32)
    _, com, vm, sg = oracle.halo_props(pos, vel, hid, 1, 10.0)
    w = 0.7
    gp, gv = oracle.halo_props_backward(vel, hid, 1, vm, sg, g_com=2 * w * com,
                                        g_sigv=np.array([2 * w * sg[0]]))
    assert np.allclose(gp, 2 * w * com[0] / n, rtol=1e-12)
    assert np.allclose(gv, 2 * w * (vel - vm[0]) / (3 * n), rtol=1e-12)


# --------------------------------------------------------------------------
# REINFORCE pieces (Sec. 3.2, Eqs. 6-8)

def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert oracle.philox4x32_10(v[0:4], v[4:6]).tolist() == v[6:10]


def test_exp_within_2ulp_of_fp64():
    xs = np.concatenate([np.linspace(-87, 87, 40001, dtype=np.float32),
                         np.array([0.0, -0.0, 1e-30, -1e-30, 0.5 * math.log(2)], np.float32)])
    for x in xs:
        e = oracle.exp32(float(x))
        t = math.exp(float(x))
        assert abs(e - t) <= 2 * float(np.spacing(np.float32(t))), x
    assert oracle.exp32(200.0) == oracle.exp32(87.0)
    assert oracle.exp32(-200.0) == oracle.exp32(-87.0)


def test_edge_prob_forms():
    b = 0.3125
    # form 0: sigma((b-d)/tau), tau = 0.05 b: p(b) = 1/2, decreasing in d
    coef = oracle.prob_coef(b, 0)
    assert oracle.edge_prob(b, b * b, b, 0, coef) == 0.5
    d = 0.9 * b
    z = (b - d) / (0.05 * b)
    assert abs(oracle.edge_prob(d, d * d, b, 0, coef) - 1 / (1 + math.exp(-z))) < 1e-6
    # form 1 (Eq. 8): sigma(alpha (b2 - d2)/b2)
    c1 = oracle.prob_coef(b, 1, alpha=5.0)
    d = 1.2 * b
    z = 5.0 * (b * b - d * d) / (b * b)
    assert abs(oracle.edge_prob(d, d * d, b, 1, c1) - 1 / (1 + math.exp(-z))) < 1e-6


def test_pairs_match_brute_force():
    N, L = 1500, 6.0
    pos = synth.uniform(N, L, 9).numpy()
    b = 0.3
    rc = float(np.float32(1.5 * np.float32(b)))
    pi, pj, pd, pp = oracle.pairs(pos, L, b, rc, 0, oracle.prob_coef(b, 0))
    rc2 = np.float32(rc) * np.float32(rc)
    exp = []
    for i in range(N):
        for j in range(i + 1, N):
            if np.float32(oracle.dist2(pos[i], pos[j], L)) < rc2:
                exp.append((i, j))
    assert list(zip(pi.tolist(), pj.tolist())) == exp
    assert np.all(pd == np.sqrt(np.float32([oracle.dist2(pos[i], pos[j], L) for i, j in exp])))
    assert ((pp > 0) & (pp <= 1)).all()


def test_edge_uniform_unbiased_and_link_frequency():
    # u is uniform in [0,1): link frequency of an edge over samples ~ Bernoulli(p)
    K = 20000
    us = np.array([oracle.edge_uniform(123, 7, 3, k) for k in range(K)])
    assert us.min() >= 0 and us.max() < 1
    assert abs(us.mean() - 0.5) < 4 * math.sqrt(1 / 12 / K)
    # symmetric in (i, j)
    assert oracle.edge_uniform(5, 2, 9, 3) == oracle.edge_uniform(5, 9, 2, 3)
    p = 0.3
    freq = (us < p).mean()
    assert abs(freq - p) < 4 * math.sqrt(p * (1 - p) / K)
    # chi-square over 16 bins
    h, _ = np.histogram(us, bins=16, range=(0, 1))
    chi2 = ((h - K / 16) ** 2 / (K / 16)).sum()
    assert chi2 < 50  # 15 dof, p ~ 1e-5


def _tiny_graph():
    pos = np.array([[1.0, 1.0, 1.0], [1.28, 1.0, 1.0], [1.1, 1.3, 1.0],
                    [1.5, 1.2, 1.1], [1.3, 1.05, 1.35]], np.float32)
    return pos, 10.0, 0.3


def _exact_expectation(pos64, L, b, pi, pj, form, coef, loss):
    # enumerate all 2^E topologies with FP64 probabilities from the same formula
    N = pos64.shape[0]
    ps = []
    for i, j in zip(pi, pj):
        dx = (pos64[j] - pos64[i] + L / 2) % L - L / 2
        d2 = float(np.dot(dx, dx))
        d = math.sqrt(d2)
        z = (b - d) * coef if form == 0 else (b * b - d2) * coef
        ps.append(1 / (1 + math.exp(-z)))
    E = len(ps)
    tot = 0.0
    for ys in itertools.product([0, 1], repeat=E):
        pr = 1.0
        par = list(range(N))

        def f(x):
            while par[x] != x:
                x = par[x]
            return x
        for e, y in enumerate(ys):
            pr *= ps[e] if y else 1 - ps[e]
            if y:
                a, c = f(pi[e]), f(pj[e])
                if a != c:
                    par[max(a, c)] = min(a, c)
        labs = [f(i) for i in range(N)]
        tot += pr * loss(labs)
    return tot


def test_reinforce_gradient_unbiased_exact_enumeration():
    pos, L, b = _tiny_graph()
    form = 0
    coef = float(oracle.prob_coef(b, form))
    rc = float(np.float32(1.5 * np.float32(b)))
    pi, pj, pd, pp = oracle.pairs(pos, L, b, rc, form, coef)
    E = len(pi)
    assert 5 <= E <= 10

    def loss(labs):  # number of groups with >= 2 members
        from collections import Counter
        return sum(1 for v in Counter(labs).values() if v >= 2)

    pos64 = pos.astype(np.float64)
    exact = np.zeros((5, 3))
    h = 1e-5
    for i in range(5):
        for a in range(3):
            pos64[i, a] += h
            fp = _exact_expectation(pos64, L, b, pi, pj, form, coef, loss)
            pos64[i, a] -= 2 * h
            fm = _exact_expectation(pos64, L, b, pi, pj, form, coef, loss)
            pos64[i, a] += h
            exact[i, a] = (fp - fm) / (2 * h)
    K = 40000
    labels, _ = oracle.reinforce_sample(5, pi, pj, pp, K, 99, 2)
    Ls = np.array([loss(l.tolist()) for l in labels], np.float64)
    A = Ls - Ls.mean()
    g = oracle.reinforce_grad(pos, L, pi, pj, pp, K, 99, A, form, coef)
    # standard error per component from per-sample contributions (batches)
    nb = 40
    parts = []
    for s in range(nb):
        sl = slice(s * K // nb, (s + 1) * K // nb)
        lb, _ = labels[sl], None
        Ab = Ls[sl] - Ls.mean()
        parts.append(_grad_from_samples(pos, L, pi, pj, pp, 99, Ab, form, coef, s * K // nb))
    se = np.std(parts, axis=0, ddof=1) / math.sqrt(nb)
    assert np.all(np.abs(g - exact) <= 4 * se + 1e-9), (g, exact, se)
    assert np.abs(exact).max() > 0.05  # the pin is not vacuous


def _grad_from_samples(pos, L, pi, pj, pp, seed, A, form, coef, k0):
    # same estimator as the oracle, restricted to samples k0..k0+len(A)-1
    N = pos.shape[0]
    g = np.zeros((N, 3))
    pos64 = pos.astype(np.float64)
    for e, (i, j) in enumerate(zip(pi, pj)):
        s = 0.0
        for t, a in enumerate(A):
            y = 1.0 if oracle.edge_uniform(seed, int(i), int(j), k0 + t) < pp[e] else 0.0
            s += a * (y - float(pp[e]))
        s /= len(A)
        dx = (pos64[j] - pos64[i] + L / 2) % L - L / 2
        d = math.sqrt(float(np.dot(dx, dx)))
        fac = coef / d if form == 0 else 2 * coef
        g[i] += s * fac * dx
        g[j] -= s * fac * dx
    return g


def test_reinforce_sample_matches_plain_fof_when_p_is_step():
    # with probability forced to {0,1} by a steep logistic, sampled FoF = plain FoF
    spec = synth.BoxSpec("t", 1500, 20.0, synth.linking_length(20.0, 1500) * 1.5, 15, 0.5, 8)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    b = spec.b
    rc = float(np.float32(1.5 * np.float32(b)))
    pi, pj, pd, pp = oracle.pairs(pos, spec.L, b, rc, 0, 1e9 / b)
    labels, nh = oracle.reinforce_sample(len(pos), pi, pj, pp, 3, 0, 20)
    ref = oracle.fof_labels(pos, spec.L, b)
    # p = 1 when d < b by a margin and p < 1e-30 when d > b; no pair sits in the
    # narrow band around d = b where the steep logistic is not saturated
    assert np.all(np.abs(pd - np.float32(b)) > 1e-6 * b)
    assert np.all((pp == 1.0) | (pp < 1e-30))
    for k in range(3):
        assert np.array_equal(labels[k], ref)
    _, cnt = oracle.groups(ref, 20)
    assert (nh == len(cnt)).all()


# --------------------------------------------------------------------------
# Restricted helpers used by the full-size checks (Sec. 3.2, Eqs. 6-8): each
# must equal the unrestricted function it restricts, which the pins above fix.

def _reinforce_box():
    spec = synth.BoxSpec("t", 3000, 24.0, synth.linking_length(24.0, 3000) * 1.3, 30, 0.6, 11)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    b = spec.b
    rc = float(np.float32(1.5 * np.float32(b)))
    coef = oracle.prob_coef(b, 0)
    pi, pj, pd, pp = oracle.pairs(pos, spec.L, b, rc, 0, coef)
    assert len(pi) > 2000
    return spec, pos, pi, pj, pp, coef


def test_reinforce_sample_one_is_a_row_of_the_full_sample():
    spec, pos, pi, pj, pp, _ = _reinforce_box()
    K, seed = 9, 0x5EED  # K not a multiple of the four samples one Philox call serves
    labels, nh = oracle.reinforce_sample(spec.N, pi, pj, pp, K, seed, 5)
    rows = set()
    for k in range(K):
        lab, h = oracle.reinforce_sample_one(spec.N, pi, pj, pp, k, seed, 5)
        assert np.array_equal(lab, labels[k]), k
        assert h == nh[k], k
        rows.add(lab.tobytes())
    assert len(rows) == K  # every sample differs: a wrong sample index fails
    # a different seed draws different samples
    lab0, _ = oracle.reinforce_sample_one(spec.N, pi, pj, pp, 0, seed + 1, 5)
    assert not np.array_equal(lab0, labels[0])


def test_reinforce_grad_masked_restricts_the_full_gradient():
    spec, pos, pi, pj, pp, coef = _reinforce_box()
    K, seed = 12, 77
    A = np.random.default_rng(4).standard_normal(K)
    A -= A.mean()
    for form, c in ((0, coef), (1, oracle.prob_coef(spec.b, 1, alpha=0.5))):
        full = oracle.reinforce_grad(pos, spec.L, pi, pj, pp, K, seed, A, form, c)
        assert np.abs(full).max() > 0
        ones = np.ones(spec.N, np.uint8)
        g1 = oracle.reinforce_grad_masked(pos, spec.L, pi, pj, pp, K, seed, A, form, c, ones)
        assert np.array_equal(g1, full)
        # a mask that splits many pairs: rows inside equal the full rows
        # (their partners outside still contribute), rows outside stay 0
        mask = (np.random.default_rng(5).random(spec.N) < 0.5).astype(np.uint8)
        inside = mask.astype(bool)
        split = np.count_nonzero(inside[pi] != inside[pj])
        assert split > 100
        gm = oracle.reinforce_grad_masked(pos, spec.L, pi, pj, pp, K, seed, A, form, c, mask)
        assert np.array_equal(gm[inside], full[inside])
        assert not gm[~inside].any()


# --------------------------------------------------------------------------
# Decorated frozen assignment and the soft-histogram mass function
# (Sec. 3.1.1, Eq. 5): the decoration D_h (particle standard deviation about
# the halo centre), its adjoint, the soft histogram and its VJP.

def test_decoration_closed_form_across_the_boundary():
    L, a = 10.0, 0.3
    c = np.array([0.05, 9.9, 4.0])  # straddles two periodic faces
    off = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, a], [0, 0, -a]])
    pos = (c + off) % L
    hid = np.zeros(6, np.int32)
    _, com, _, _ = oracle.halo_props(pos, np.zeros_like(pos), hid, 1, L)
    assert np.allclose(com[0], c, atol=1e-12)
    D = oracle.halo_decoration(pos, hid, 1, L, com)
    assert abs(D[0] - a / math.sqrt(3.0)) < 1e-12


def _decor_box(seed=3):
    rng = np.random.default_rng(seed)
    L = 20.0
    centres = rng.uniform(0, L, (3, 3))
    centres[0] = [0.1, 19.95, 10.0]  # one halo across the faces
    sizes = [7, 12, 25]
    pos = np.concatenate([(cc + rng.normal(0, 0.2, (m, 3))) % L for cc, m in zip(centres, sizes)]
                         + [rng.uniform(0, L, (10, 3))])
    hid = np.concatenate([np.full(m, h, np.int32) for h, m in enumerate(sizes)] + [np.full(10, -1, np.int32)])
    return pos, hid, L, 3


def _decor_of(pos, hid, H, L):
    _, com, _, _ = oracle.halo_props(pos, np.zeros_like(pos), hid, H, L)
    return oracle.halo_decoration(pos, hid, H, L, com), com


def test_decoration_backward_matches_central_differences():
    # the adjoint drops the centre's dependence on x (its deviations sum to
    # zero); central differences move the centre too
    pos, hid, L, H = _decor_box()
    D, com = _decor_of(pos, hid, H, L)
    g_dsig = np.array([0.7, -1.3, 2.1])
    g = oracle.halo_decoration_backward(pos, hid, H, L, com, D, g_dsig)
    eps = 1e-6
    fd = np.zeros_like(pos)
    for i in range(pos.shape[0]):
        for a in range(3):
            p1 = pos.copy(); p1[i, a] += eps
            p0 = pos.copy(); p0[i, a] -= eps
            fd[i, a] = (g_dsig @ _decor_of(p1, hid, H, L)[0] - g_dsig @ _decor_of(p0, hid, H, L)[0]) / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)
    assert not g[hid < 0].any()


def test_soft_hist_limits_and_vjp():
    rng = np.random.default_rng(4)
    ell = rng.uniform(1.0, 9.0, 400)
    edges = np.linspace(0.0, 10.0, 11)
    ell = ell[np.min(np.abs(ell[:, None] - edges[None, :]), 1) > 1e-3]  # none on an edge
    hard, _ = np.histogram(ell, bins=edges)
    assert np.allclose(oracle.soft_hist(ell, edges, 1e-5), hard, atol=1e-9)
    soft = oracle.soft_hist(ell, edges, 0.3)
    # the bins telescope: their sum only sees the outer edges
    S = lambda t: 1.0 / (1.0 + np.exp(-t))
    assert abs(soft.sum() - (S((ell - edges[0]) / 0.3) - S((ell - edges[-1]) / 0.3)).sum()) < 1e-9
    g_hist = rng.normal(size=10)
    g = oracle.soft_hist_backward(ell, edges, 0.3, g_hist)
    eps = 1e-6
    for h in range(0, len(ell), 37):
        e1 = ell.copy(); e1[h] += eps
        e0 = ell.copy(); e0[h] -= eps
        fd = (g_hist @ oracle.soft_hist(e1, edges, 0.3) - g_hist @ oracle.soft_hist(e0, edges, 0.3)) / (2 * eps)
        assert abs(g[h] - fd) < 1e-6 * max(1.0, abs(fd))


def surrogate_log_mass(counts, D, D0, kappa, particle_mass=1.0):
    """Decorated log-mass: log(m_p n_h) in value; its derivative follows the
    decoration with weight -kappa (sigma as an inverse mass proxy)."""
    return np.log(particle_mass * np.asarray(counts, np.float64)) - kappa * (np.log(D) - np.log(D0))


def test_decorated_mass_function_gradient_chain():
    # d/dx sum_k g_k H_k(ell(D(x))) with D0 frozen: the chain of the two
    # adjoints, g_D = -kappa g_ell / D, equals central differences
    pos, hid, L, H = _decor_box(5)
    counts = np.bincount(hid[hid >= 0], minlength=H)
    D0, com = _decor_of(pos, hid, H, L)
    edges = np.log(np.array([4.0, 8.0, 16.0, 32.0]))
    kappa, w = 1.5, 0.4
    g_hist = np.array([0.3, -1.0, 0.8])

    def loss(p):
        D, _ = _decor_of(p, hid, H, L)
        return g_hist @ oracle.soft_hist(surrogate_log_mass(counts, D, D0, kappa), edges, w)

    ell = surrogate_log_mass(counts, D0, D0, kappa)
    g_ell = oracle.soft_hist_backward(ell, edges, w, g_hist)
    g = oracle.halo_decoration_backward(pos, hid, H, L, com, D0, -kappa * g_ell / D0)
    eps = 1e-6
    for i in range(0, pos.shape[0], 3):
        for a in range(3):
            p1 = pos.copy(); p1[i, a] += eps
            p0 = pos.copy(); p0[i, a] -= eps
            fd = (loss(p1) - loss(p0)) / (2 * eps)
            assert abs(g[i, a] - fd) < 1e-6 * max(1.0, abs(fd)), (i, a)
    assert np.abs(g).max() > 1e-3


# --------------------------------------------------------------------------
# Sub-halos: FoF in phase space inside each halo (Sec. 2.1.1, Eq. 3)

def _halos_of(pos, L, b, min_size):
    lab = oracle.fof_labels(pos, L, b)
    hid, cnt = oracle.groups(lab, min_size)
    return hid, len(cnt)


def _subhalo_reference_by_position(pos, hid, H, L, b):
    # per halo: brute-force FoF of its members alone, local labels -> indices
    out = np.arange(pos.shape[0], dtype=np.int32)
    for h in range(H):
        m = np.nonzero(hid == h)[0]
        loc = oracle.fof_brute(pos[m], L, b)
        out[m] = m[loc]
    return out


def test_subhalo_equal_velocities_is_fof_of_each_halo():
    # identical velocities and sigma_x = 1/4 (1/sigma_x = 4 exactly): the
    # phase-space test is exactly d2 <= (1/2)^2, so each halo splits as the
    # brute-force FoF of its members with b = 1/2
    spec = synth.BoxSpec("t", 4000, 30.0, 1.0, 25, 0.7, 6)
    pos, _ = synth.generate(spec, velocities=False)
    pos = pos.numpy()
    hid, H = _halos_of(pos, spec.L, 1.0, 10)
    assert H > 5
    vel = np.tile(np.float32([3.0, -2.0, 5.0]), (pos.shape[0], 1))
    got = oracle.subhalo_labels(pos, vel, hid, H, spec.L, 0.25, 1.0)
    want = _subhalo_reference_by_position(pos, hid, H, spec.L, 0.5)
    assert np.array_equal(got, want)
    assert len(set(got[hid >= 0].tolist())) > H  # the halos do split
    # an infinite velocity scale switches the velocity term off
    vel2 = np.random.default_rng(1).normal(0, 100, pos.shape).astype(np.float32)
    assert np.array_equal(oracle.subhalo_labels(pos, vel2, hid, H, spec.L, 0.25, np.inf), want)


def test_subhalo_splits_coincident_streams():
    # two interpenetrating clumps, one halo in position, two in phase space
    rng = np.random.default_rng(7)
    L = 20.0
    a = 10.0 + rng.normal(0, 0.05, (300, 3))
    b = 10.0 + rng.normal(0, 0.05, (300, 3))
    pos = np.concatenate([a, b]).astype(np.float32)
    vel = np.concatenate([np.tile([200.0, 0, 0], (300, 1)) + rng.normal(0, 1, (300, 3)),
                          np.tile([-200.0, 0, 0], (300, 1)) + rng.normal(0, 1, (300, 3))]).astype(np.float32)
    perm = rng.permutation(600)
    pos, vel = pos[perm], vel[perm]
    hid, H = _halos_of(pos, L, 0.1, 20)
    assert H == 1 and (hid == 0).all()
    sub = oracle.subhalo_labels(pos, vel, hid, H, L, 0.2 ** 2, 20.0 ** 2)
    stream = (vel[:, 0] > 0)
    assert len(set(sub[stream].tolist())) == 1 and len(set(sub[~stream].tolist())) == 1
    assert sub[stream][0] != sub[~stream][0]
    assert sub[stream][0] == np.nonzero(stream)[0].min()


def test_subhalo_invariants_on_a_clustered_box():
    spec = synth.BoxSpec("t", 6000, 25.0, synth.linking_length(25.0, 6000) * 1.3, 40, 0.7, 9)
    pos, vel = synth.generate(spec)
    pos, vel = pos.numpy(), vel.numpy()
    hid, H = _halos_of(pos, spec.L, spec.b, 20)
    sx, sv = (0.5 * spec.b) ** 2, 40.0 ** 2
    sub = oracle.subhalo_labels(pos, vel, hid, H, spec.L, sx, sv)
    inv_sx, inv_sv = np.float32(1 / sx), np.float32(1 / sv)

    def d2(i, j):
        return oracle.dist2(pos[i], pos[j], spec.L) * inv_sx + float(np.sum((vel[j] - vel[i]) ** 2)) * inv_sv

    N = pos.shape[0]
    assert np.all(sub[hid < 0] == np.nonzero(hid < 0)[0])
    for h in range(H):
        m = np.nonzero(hid == h)[0]
        assert np.all(hid[sub[m]] == h) and np.all(sub[m] <= m)  # inside the halo, smallest member
        for g in np.unique(sub[m]):
            grp = m[sub[m] == g]
            assert g == grp.min()
            rest = m[sub[m] != g]
            for i in grp[:20]:
                # no member outside the group is a phase-space friend (with a margin)
                assert all(d2(i, j) > 1.0 + 1e-5 for j in rest[:200])
    assert len(np.unique(sub[hid >= 0])) > H
