"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Labels, halo ids, counts and CSR members must be
bit-exact; properties and adjoints within the stated tolerances."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Tolerances (FP32 compensated sums against the FP64 oracle):
COM_TOL = 1e-5      # periodic COM error as a fraction of L
SIGV_RTOL = 1e-4    # velocity dispersion, relative
VMEAN_TOL = 1e-5    # |vmean error| / mean |v| of the halo
BWD_RTOL = 1e-4     # adjoint vs analytic FP64 adjoint, relative (with an absolute floor)


@pytest.fixture(scope="module")
def J():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26851_gb300 import build
    build.build()
    import paper_2510_26851_gb300 as j
    return j


def run_fof(J, pos_np, L, b, min_size=20, n_axis=0, wrap=False):
    pos = torch.from_numpy(np.ascontiguousarray(pos_np, np.float32)).cuda()
    r = J.fof(pos, L, b, min_size=min_size, n_axis=n_axis, wrap=wrap)
    J.sync()
    H = r.groups.n_halos
    return pos, r, H


def check_groups(r, H, lab_ref, min_size):
    hid_ref, cnt_ref = oracle.groups(lab_ref, min_size)
    assert H == len(cnt_ref)
    assert np.array_equal(r.groups.halo_id.cpu().numpy(), hid_ref)
    assert np.array_equal(r.groups.count[:H].cpu().numpy(), cnt_ref)
    hs = r.groups.halo_start[:H + 1].cpu().numpy()
    assert hs[0] == 0 and np.array_equal(np.diff(hs), cnt_ref)
    mem = r.groups.members[:hs[-1]].cpu().numpy()
    order = np.argsort(hid_ref[hid_ref >= 0], kind="stable")
    expect = np.nonzero(hid_ref >= 0)[0][order]
    assert np.array_equal(mem, expect)
    return hid_ref, cnt_ref


def test_hand_cases(J):
    for c in json.load(open(os.path.join(GOLDEN, "fof_hand_cases.json")))["cases"]:
        pos = np.array(c["pos"], np.float32)
        _, r, _ = run_fof(J, pos, c["L"], c["b"], min_size=1)
        assert r.label.cpu().tolist() == c["labels"], c["name"]


def test_small_clustered_box_bit_exact(J):
    spec = synth.SMALL_32
    pos, _ = synth.generate(spec, device="cuda")
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    _, r, H = run_fof(J, pos_np, spec.L, spec.b, spec.min_size)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    check_groups(r, H, lab_ref, spec.min_size)
    assert H > 50


@pytest.mark.parametrize("seed", [0, 1])
def test_labels_invariant_across_grids(J, seed):
    N, L = 20000, 20.0
    pos_np = synth.uniform(N, L, seed).numpy()
    b = 0.8 * L / N ** (1 / 3)
    lab_ref = oracle.fof_labels(pos_np, L, b)
    nmax = J.max_cells_per_axis(L, b)
    for n in sorted({1, 3, 4, 7, 16, 17, 33, nmax}):
        if n > nmax:
            continue
        _, r, _ = run_fof(J, pos_np, L, b, 1, n_axis=n)
        assert np.array_equal(r.label.cpu().numpy(), lab_ref), n


def test_both_binning_paths(J):
    # grids of at most 4096 bricks (16^3 cells each) bin with the per-CTA
    # counting sort, larger ones with brick cursors: n = 256 and n = 257 sit on
    # either side of that switch; the default and the largest grid as well
    spec = synth.BoxSpec("t", 300_000, 100.0, synth.linking_length(100.0, 300_000), 1500, 0.55, 11)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    nmax = J.max_cells_per_axis(spec.L, spec.b)
    assert nmax > 257
    for n in (0, 256, 257, nmax):
        _, r, H = run_fof(J, pos_np, spec.L, spec.b, spec.min_size, n_axis=n)
        assert np.array_equal(r.label.cpu().numpy(), lab_ref), n
        check_groups(r, H, lab_ref, spec.min_size)


@pytest.mark.parametrize("boost", [1.0, 2.5])
def test_labels_invariant_across_cell_classes(J, boost):
    # dense threshold 0 turns the sub-cell path off; 1 sends almost every cell
    # through it; small threshold 0 sends every cell to the warp paths
    spec = synth.BoxSpec("t", 300_000, 67.0, synth.linking_length(67.0, 300_000) * boost, 1500, 0.6, 9)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    n = J.default_cells_per_axis(spec.N, spec.L, spec.b)
    ic = np.minimum((pos_np.astype(np.float64) * (n / spec.L)).astype(np.int64), n - 1)
    m = np.bincount(ic[:, 0] + n * (ic[:, 1] + n * ic[:, 2]), minlength=n ** 3)
    assert ((m > 96) & (m <= 160)).any() and (m > 160).any()  # both large-medium paths are used
    try:
        # (16, 160): the large-box default; (16, 128), (24, 200): medium cells of
        # 97-160 particles on their own bitmask and list paths, larger ones on
        # the shared-memory union-find
        for S, T in ((0, 0), (0, 1), (8, 0), (1, 8), (8, 64), (3, 12), (64, 1000), (100000, 0), (16, 160),
                     (16, 128), (24, 200), (16, -1)):
            J.set_cell_classes(S, T)
            _, r, H = run_fof(J, pos_np, spec.L, spec.b, spec.min_size)
            assert np.array_equal(r.label.cpu().numpy(), lab_ref), (S, T)
    finally:
        J.set_cell_classes()


def test_ragged_sizes_and_tiny_boxes(J):
    rng = np.random.default_rng(0)
    for N in (1, 2, 3, 31, 33, 255, 257, 4097):
        L = 5.0
        pos_np = rng.uniform(0, L, (N, 3)).astype(np.float32)
        pos_np[pos_np >= L] = 0
        b = 0.9 * L / max(N, 8) ** (1 / 3)
        lab_ref = oracle.fof_brute(pos_np, L, b)
        _, r, H = run_fof(J, pos_np, L, b, 2)
        assert np.array_equal(r.label.cpu().numpy(), lab_ref), N
        check_groups(r, H, lab_ref, 2)


def test_lattice_closed_forms(J):
    m = 16
    idx = np.arange(m, dtype=np.float32)
    gz, gy, gx = np.meshgrid(idx, idx, idx, indexing="ij")
    pos_np = np.stack([gx, gy, gz], -1).reshape(-1, 3).astype(np.float32)
    L = float(m)
    _, r, H = run_fof(J, pos_np, L, 1.0 / 0.9, 20)
    assert (r.label.cpu().numpy() == 0).all() and H == 1
    assert r.groups.count[0].item() == m ** 3
    assert np.array_equal(r.groups.members[:m ** 3].cpu().numpy(), np.arange(m ** 3))
    _, r, H = run_fof(J, pos_np, L, 1.0 / 1.1, 1)
    assert np.array_equal(r.label.cpu().numpy(), np.arange(m ** 3)) and H == m ** 3


def test_member_segments_of_every_length(J):
    # fully linked clumps (side 0.2 < b / sqrt(3)) far apart, with sizes on
    # both sides of every boundary of the segmented sort: one warp in
    # registers up to 256 (32, 64, 128 per network size), one block in shared
    # memory up to 8192, chunks beyond; input order shuffled so each halo's
    # members arrive unsorted
    rng = np.random.default_rng(7)
    sizes = [1, 2, 3, 31, 32, 33, 64, 65, 128, 129, 255, 257, 511, 513, 1000, 1024, 1025, 2047, 2049,
             4096, 8192, 8193, 12000]
    L, b = 100.0, 0.5
    pts = []
    for t, n in enumerate(sizes):
        c = np.array([5.0 + 9.0 * (t % 10), 5.0 + 9.0 * ((t // 10) % 10), 50.0])
        pts.append(c + rng.uniform(0.0, 0.2, (n, 3)))
    pos_np = np.concatenate(pts).astype(np.float32)
    pos_np = pos_np[rng.permutation(len(pos_np))]
    lab_ref = oracle.fof_labels(pos_np, L, b)
    _, r, H = run_fof(J, pos_np, L, b, 1)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    check_groups(r, H, lab_ref, 1)
    assert H == len(sizes)


def test_split_entry_points_bin_link_groups(J):
    # jfof_bin_cells -> jfof_link (labels only, through the bucketed scatter)
    # -> jfof_groups (groups of given labels): the oracle's labels and groups;
    # 300k particles take 74 scatter buckets of 4096, 4.5M the 1024-bucket
    # limit with wider buckets
    import types
    for N, L, nh, seed in ((300_000, 67.0, 1500, 21), (4_500_000, 160.0, 25_000, 22)):
        spec = synth.BoxSpec("t", N, L, synth.linking_length(L, N), nh, 0.6, seed, velocities=False)
        pos, _ = synth.generate(spec, device="cuda", velocities=False)
        pos_np = pos.cpu().numpy()
        lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
        grid = J.bin_cells(pos, spec.L, spec.b)
        lab = J.link(grid)
        J.sync()
        assert np.array_equal(lab.cpu().numpy(), lab_ref)
        g = J.groups(lab, spec.min_size)
        J.sync()
        check_groups(types.SimpleNamespace(groups=g), g.n_halos, lab_ref, spec.min_size)
        g2 = J.groups(torch.from_numpy(lab_ref).cuda(), spec.min_size)
        J.sync()
        check_groups(types.SimpleNamespace(groups=g2), g2.n_halos, lab_ref, spec.min_size)


def test_wrap_flag_and_boundary(J):
    rng = np.random.default_rng(4)
    N, L, b = 30000, 12.0, 0.25
    p = rng.uniform(-L, 2 * L, (N, 3)).astype(np.float32)
    wrapped = oracle.wrap(p, L)
    lab_ref = oracle.fof_labels(wrapped, L, b)
    _, r, _ = run_fof(J, p, L, b, 1, wrap=True)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)


def test_out_of_range_latches_erange(J):
    p = np.array([[1.0, 2.0, 3.0], [1.1, 2.0, 12.5]], np.float32)
    pos = torch.from_numpy(p).cuda()
    J.fof(pos, 10.0, 0.5, min_size=1)
    with pytest.raises(J.JfofError) as e:
        J.sync()
    assert e.value.code == J.JFOF_ERANGE
    J.sync()  # cleared


def test_bad_arguments_rejected_on_host(J):
    pos = torch.zeros(4, 3, device="cuda")
    with pytest.raises(J.JfofError):
        J.fof(pos, 10.0, 6.0)  # b >= L/2
    with pytest.raises(J.JfofError):
        J.fof(pos, 10.0, 0.5, n_axis=2)


def test_union_find_budget_timeout_is_reported(J):
    # a budget of one CAS retry per union cannot finish a dense cluster: the
    # bounded loop gives up, latches JFOF_ETIMEOUT and returns
    rng = np.random.default_rng(1)
    p = (5.0 + rng.normal(0, 0.05, (20000, 3))).astype(np.float32)
    pos = torch.from_numpy(p).cuda()
    J.set_loop_budget(1)
    try:
        J.fof(pos, 10.0, 0.3, min_size=1)
        with pytest.raises(J.JfofError) as e:
            J.sync()
        assert e.value.code == J.JFOF_ETIMEOUT
    finally:
        J.set_loop_budget(0)
    J.fof(pos, 10.0, 0.3, min_size=1)
    J.sync()


def props_check(J, pos, vel, r, H, L, lab_ref, min_size):
    hid_ref, cnt_ref = oracle.groups(lab_ref, min_size)
    p = J.halo_props(pos, vel, L, r.groups, particle_mass=1.0)
    J.sync()
    pos64 = pos.cpu().numpy().astype(np.float64)
    vel64 = vel.cpu().numpy().astype(np.float64)
    m_ref, com_ref, vm_ref, sg_ref = oracle.halo_props(pos64, vel64, hid_ref, H, L)
    assert np.array_equal(p.mass[:H].cpu().numpy(), m_ref.astype(np.float32))
    com = p.com[:H].cpu().numpy().astype(np.float64)
    dcom = np.abs((com - com_ref + L / 2) % L - L / 2) / L
    assert dcom.max() <= COM_TOL, dcom.max()
    assert ((com >= 0) & (com < L)).all()
    sg = p.sigv[:H].cpu().numpy()
    assert (np.abs(sg - sg_ref) <= SIGV_RTOL * np.abs(sg_ref) + 1e-30).all()
    vm = p.vmean[:H].cpu().numpy()
    absv = np.zeros(H)
    np.add.at(absv, hid_ref[hid_ref >= 0], np.abs(vel64[hid_ref >= 0]).mean(1))
    scale = absv / cnt_ref
    assert (np.abs(vm - vm_ref).max(1) <= VMEAN_TOL * scale + 1e-6).all()
    return p, hid_ref, cnt_ref, (m_ref, com_ref, vm_ref, sg_ref)


def test_props_and_backward_clustered_box(J):
    spec = synth.BoxSpec("t", 200_000, 60.0, synth.linking_length(60.0, 200_000), 1200, 0.6, 5)
    pos, vel = synth.generate(spec, device="cuda")
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    _, r, H = run_fof(J, pos_np, spec.L, spec.b, spec.min_size)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    p, hid_ref, cnt_ref, ref = props_check(J, pos, vel, r, H, spec.L, lab_ref, spec.min_size)
    # adjoint with the C5a loss: g_com = 2 w com, g_sigv = 2 w sigma
    w = torch.rand(H, generator=torch.Generator().manual_seed(1), dtype=torch.float64).numpy()
    g_com = torch.zeros(r.groups.H_cap, 3, device="cuda")
    g_sig = torch.zeros(r.groups.H_cap, device="cuda")
    g_com[:H] = torch.from_numpy(2 * w[:, None] * p.com[:H].cpu().numpy()).float().cuda()
    g_sig[:H] = torch.from_numpy(2 * w * p.sigv[:H].cpu().numpy()).float().cuda()
    gp, gv = J.halo_props_backward(vel, r.groups, p.vmean, p.sigv, g_com=g_com, g_sigv=g_sig)
    J.sync()
    gp_ref, gv_ref = oracle.halo_props_backward(
        vel.cpu().numpy().astype(np.float64), hid_ref, H, p.vmean[:H].cpu().numpy(),
        p.sigv[:H].cpu().numpy(), g_com=g_com[:H].cpu().numpy(), g_sigv=g_sig[:H].cpu().numpy())
    for got, want in ((gp.cpu().numpy(), gp_ref), (gv.cpu().numpy(), gv_ref)):
        err = np.abs(got - want)
        assert (err <= BWD_RTOL * np.abs(want) + 1e-6 * np.abs(want).max()).all(), err.max()


def test_props_cold_halo_with_outlier_first_member(J):
    # a 2400-member cold halo (bulk ~ 1100) whose smallest-index member is a
    # velocity outlier at the halo's edge, plus a uniform background: sigma_v
    # within 1e-4 of the FP64 oracle (a one-pass sum shifted by that member
    # loses about 3n = 7200 ulp of sigma^2 here), COM within 1e-5 L
    from test_oracle import _cold_halo_with_outlier
    hp, hv, L = _cold_halo_with_outlier()
    rng = np.random.default_rng(3)
    nb = 40_000
    bp = rng.uniform(0, L, (nb, 3)).astype(np.float32)
    bv = rng.normal(0, 300, (nb, 3)).astype(np.float32)
    pos_np = np.concatenate([hp, bp])
    vel_np = np.concatenate([hv, bv])
    b = float(np.float32(0.2 * L / (len(pos_np) ** (1 / 3))))
    lab_ref = oracle.fof_labels(pos_np, L, b)
    pos, r, H = run_fof(J, pos_np, L, b, 20)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    assert np.all(lab_ref[:len(hp)] == 0)  # the halo is one group, led by the outlier
    props_check(J, pos, torch.from_numpy(vel_np).cuda(), r, H, L, lab_ref, 20)


def test_autograd_function(J):
    spec = synth.BoxSpec("t", 50_000, 40.0, synth.linking_length(40.0, 50_000), 300, 0.6, 6)
    pos, vel = synth.generate(spec, device="cuda")
    r = J.fof(pos, spec.L, spec.b, spec.min_size)
    pos = pos.clone().requires_grad_(True)
    vel = vel.clone().requires_grad_(True)
    com, vm, sg = J.HaloProps.apply(pos, vel, r.groups, spec.L)
    H = com.shape[0]
    w = torch.rand(H, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    loss = (w * ((com ** 2).sum(1) + sg ** 2)).sum()
    loss.backward()
    J.sync()
    hid = r.groups.halo_id.long()
    cnt = r.groups.count[:H].float()
    mem = hid >= 0
    exp_gp = torch.zeros_like(pos)
    exp_gp[mem] = (2 * w[:, None] * com.detach() / cnt[:, None])[hid[mem]]
    exp_gv = torch.zeros_like(vel)
    exp_gv[mem] = (2 * w[:, None] / (3 * cnt[:, None]))[hid[mem]] * (vel.detach()[mem] - vm.detach()[hid[mem]])
    assert torch.allclose(pos.grad, exp_gp, rtol=1e-4, atol=1e-6 * exp_gp.abs().max().item())
    assert torch.allclose(vel.grad, exp_gv, rtol=1e-4, atol=1e-6 * exp_gv.abs().max().item())


def test_diff_box_128cubed_frozen_adjoint(J):
    # the 128^3 differentiable-mode box itself: labels and groups against the
    # oracle, properties within tolerance, and the adjoint of
    # L = sum_h w_h (|com_h|^2 + sigma_h^2), w_h ~ U(0,1), against the FP64
    # analytic adjoint of the oracle
    spec = synth.DIFF_128
    pos, vel = synth.generate(spec, device="cuda")
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    _, r, H = run_fof(J, pos_np, spec.L, spec.b, spec.min_size)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    check_groups(r, H, lab_ref, spec.min_size)
    p, hid_ref, cnt_ref, ref = props_check(J, pos, vel, r, H, spec.L, lab_ref, spec.min_size)
    w = np.random.default_rng(1).uniform(0.0, 1.0, H)
    g_com = torch.zeros(r.groups.H_cap, 3, device="cuda")
    g_sig = torch.zeros(r.groups.H_cap, device="cuda")
    g_com[:H] = torch.from_numpy(2 * w[:, None] * p.com[:H].cpu().numpy()).float().cuda()
    g_sig[:H] = torch.from_numpy(2 * w * p.sigv[:H].cpu().numpy()).float().cuda()
    gp, gv = J.halo_props_backward(vel, r.groups, p.vmean, p.sigv, g_com=g_com, g_sigv=g_sig)
    J.sync()
    gp_ref, gv_ref = oracle.halo_props_backward(
        vel.cpu().numpy().astype(np.float64), hid_ref, H, p.vmean[:H].cpu().numpy(),
        p.sigv[:H].cpu().numpy(), g_com=g_com[:H].cpu().numpy(), g_sigv=g_sig[:H].cpu().numpy())
    for got, want in ((gp.cpu().numpy(), gp_ref), (gv.cpu().numpy(), gv_ref)):
        err = np.abs(got - want)
        assert (err <= BWD_RTOL * np.abs(want) + 1e-6 * np.abs(want).max()).all(), err.max()


def test_box_256cubed_full_parity(J):
    spec = synth.BOX_256
    pos, vel = synth.generate(spec, device="cuda")
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    _, r, H = run_fof(J, pos_np, spec.L, spec.b, spec.min_size)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    check_groups(r, H, lab_ref, spec.min_size)
    props_check(J, pos, vel, r, H, spec.L, lab_ref, spec.min_size)


def test_host_buffer_step_matches_device_path(J):
    # jfof_fof_host (host inputs, velocity upload overlapped with the FoF
    # kernels) gives exactly jfof_fof + jfof_halo_props; page-locked and
    # pageable inputs, with and without velocities
    spec = synth.BoxSpec("t", 200_000, 60.0, synth.linking_length(60.0, 200_000), 1000, 0.6, 13)
    pos, vel = synth.generate(spec, device="cuda")
    r = J.fof(pos, spec.L, spec.b, spec.min_size)
    p = J.halo_props(pos, vel, spec.L, r.groups)
    J.sync()
    H = r.groups.n_halos
    M = int(r.groups.halo_start[H].item())  # members past M are unused
    for pinned in (True, False):
        hp, hv = pos.cpu(), vel.cpu()
        if pinned:
            hp, hv = hp.pin_memory(), hv.pin_memory()
        r2, p2, dp, dv = J.fof_host(hp, hv, spec.L, spec.b, spec.min_size)
        J.sync()
        assert torch.equal(dp, pos) and torch.equal(dv, vel)
        assert r2.groups.n_halos == H
        assert torch.equal(r2.label, r.label) and torch.equal(r2.groups.halo_id, r.groups.halo_id)
        assert torch.equal(r2.groups.halo_start[:H + 1], r.groups.halo_start[:H + 1])
        assert torch.equal(r2.groups.members[:M], r.groups.members[:M])
        for a, b in ((p2.mass, p.mass), (p2.com, p.com), (p2.vmean, p.vmean), (p2.sigv, p.sigv)):
            assert torch.equal(a[:H], b[:H])
    r3, p3, _, dv3 = J.fof_host(pos.cpu().pin_memory(), None, spec.L, spec.b, spec.min_size)
    J.sync()
    assert dv3 is None and torch.equal(r3.label, r.label)
    assert torch.equal(p3.com[:H], p.com[:H]) and torch.equal(p3.mass[:H], p.mass[:H])


def _min_image(d, L):
    return d - L * torch.round(d / L)


def _select(pos, ref, lo, hi, L, chunk=1 << 27):
    # indices of particles whose min-image offset from ref lies in [lo, hi]
    # per axis (float32, in chunks; the margins used are many ulp wide)
    out = []
    for s0 in range(0, pos.shape[0], chunk):
        rel = _min_image(pos[s0:s0 + chunk] - ref, L)
        out.append(torch.nonzero(((rel >= lo) & (rel <= hi)).all(1)).squeeze(1) + s0)
    return torch.cat(out)


def test_box_1024cubed(J):
    # The bench's workload and launch configuration (2^30 particles, default
    # grid and cell classes, jfof_fof then jfof_halo_props).  Checked by
    # properties that hold at any size, every label and halo id against the
    # threaded oracle (all cores of the host: 16 Grace cores on a GB300 machine),
    # and on sampled halos the FP64 properties.
    spec = synth.BOX_1024
    pos, vel = synth.generate(spec, device="cuda")
    r = J.fof(pos, spec.L, spec.b, spec.min_size)
    p = J.halo_props(pos, vel, spec.L, r.groups)
    J.sync()
    N, L, b = spec.N, spec.L, spec.b
    g = r.groups
    H = g.n_halos
    # labels: label[i] is the smallest index of i's group, so label <= index
    # and labels are fixed points
    lab = r.label.long()
    assert bool((lab <= torch.arange(N, device="cuda")).all())
    assert bool((lab[lab] == lab).all())
    # groups from the labels (plain torch): count per raw label, the cut,
    # halo ids ascending by raw label, CSR starts
    cnt = torch.bincount(lab, minlength=N)
    kept = cnt >= spec.min_size
    assert H == int(kept.sum())
    rank = torch.cumsum(kept, 0) - 1
    want_hid = torch.where(kept[lab], rank[lab], torch.full_like(lab, -1))
    assert torch.equal(g.halo_id.long(), want_hid)
    del want_hid, rank
    want_cnt = cnt[kept]
    assert torch.equal(g.count[:H].long(), want_cnt)
    hs = g.halo_start[:H + 1].long()
    assert int(hs[0]) == 0 and torch.equal(hs[1:] - hs[:-1], want_cnt)
    M = int(hs[H])
    assert M == int((g.halo_id >= 0).sum())
    # members: each segment holds its halo's particles, ascending
    mem = g.members[:M].long()
    seg = torch.repeat_interleave(torch.arange(H, device="cuda"), want_cnt)
    assert torch.equal(g.halo_id.long()[mem], seg)
    same = seg[1:] == seg[:-1]
    assert bool((mem[1:][same] > mem[:-1][same]).all())
    del cnt, kept, seg, same, lab
    torch.cuda.empty_cache()
    # every label and halo id against the threaded oracle (cell grid n = 1024;
    # labels do not depend on it), counts against its groups
    threads = oracle.default_threads()
    lab_ref = oracle.fof_labels_mt(pos.cpu().numpy(), L, b, n_axis=1024, threads=threads)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    hid_ref, cnt_ref = oracle.groups(lab_ref, spec.min_size)
    del lab_ref
    assert H == len(cnt_ref)
    assert np.array_equal(g.halo_id.cpu().numpy(), hid_ref)
    assert np.array_equal(g.count[:H].cpu().numpy(), cnt_ref)
    del hid_ref, cnt_ref

    rng = np.random.default_rng(7)
    counts = g.count[:H]
    picks = list(rng.choice(H, 12, replace=False)) + [int(torch.argmax(counts))]
    for h in picks:
        s0, s1 = int(hs[h]), int(hs[h + 1])
        m = mem[s0:s1]
        pm = pos[m].double()
        # neighbourhood: everything within 2 b of the halo's box (min image
        # about its first member)
        ref = pm[0]
        rel = _min_image(pm - ref, L)
        lo, hi = rel.min(0).values - 2 * b, rel.max(0).values + 2 * b
        sel = _select(pos, ref.float(), lo.float(), hi.float(), L)
        is_mem = torch.isin(sel, m)
        assert int(is_mem.sum()) == s1 - s0
        lab_s = oracle.fof_brute(pos[sel].cpu().numpy(), L, b)
        mlab = lab_s[is_mem.cpu().numpy()]
        # the members form one group, and nothing outside it links to them
        assert (mlab == mlab[0]).all(), h
        assert not (lab_s[~is_mem.cpu().numpy()] == mlab[0]).any(), h
        # FP64 properties of this halo (members in ascending index order)
        hid0 = np.zeros(s1 - s0, np.int32)
        m_ref, com_ref, vm_ref, sg_ref = oracle.halo_props(pm.cpu().numpy(), vel[m].double().cpu().numpy(),
                                                            hid0, 1, L)
        assert float(p.mass[h]) == float(m_ref[0])
        dcom = np.abs(p.com[h].double().cpu().numpy() - com_ref[0])
        dcom = np.minimum(dcom, L - dcom)
        assert (dcom <= COM_TOL * L).all(), (h, dcom)
        scale = float(vel[m].double().norm(dim=1).mean())
        assert (np.abs(p.vmean[h].double().cpu().numpy() - vm_ref[0]) <= VMEAN_TOL * scale + 1e-6).all(), h
        assert abs(float(p.sigv[h]) - sg_ref[0]) <= SIGV_RTOL * sg_ref[0] + 1e-6, h
    # random sub-cubes: particles linked inside a cube share a label
    for _ in range(8):
        c = torch.tensor(rng.uniform(0.0, L, 3), device="cuda", dtype=torch.float32)
        sel = _select(pos, c, torch.full((3,), -2.0, device="cuda"), torch.full((3,), 2.0, device="cuda"), L)
        lab_s = oracle.fof_brute(pos[sel].cpu().numpy(), L, b)
        glab = r.label[sel].cpu().numpy()
        for comp in np.unique(lab_s):
            members_c = glab[lab_s == comp]
            assert (members_c == members_c[0]).all()
    del pos, vel, r, p
    torch.cuda.empty_cache()


def test_side_stream_and_tracing(J):
    # calls enqueue on torch's current stream; with tracing on, every launch
    # is recorded under its kernel name
    spec = synth.BoxSpec("t", 150_000, 55.0, synth.linking_length(55.0, 150_000), 800, 0.6, 31, velocities=False)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    ref = J.fof(pos, spec.L, spec.b, spec.min_size)
    J.sync()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    J.trace_enable(True)
    try:
        with torch.cuda.stream(side):
            r = J.fof(pos, spec.L, spec.b, spec.min_size)
            J.sync()
            tr = J.trace_read()
    finally:
        J.trace_enable(False)
    torch.cuda.current_stream().wait_stream(side)
    assert torch.equal(r.label, ref.label)
    assert torch.equal(r.groups.halo_id, ref.groups.halo_id)
    for name in ("bin_count", "bin_scatter", "brick_sort", "link_small", "link_medium", "finalize_roots",
                 "finalize_labels", "segsort"):
        assert name in tr and tr[name][0] >= 1, (name, sorted(tr))
    assert all(t >= 0.0 for _, t in tr.values())
