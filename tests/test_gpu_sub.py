"""GPU parity for the phase-space sub-halo pass (Sec. 2.1.1, Eq. 3): sub-labels
bit-identical to the oracle's on a clustered box (several velocity scales,
the velocity term switched off, wrap), on a single large halo, and the
sub-halo groups built from them."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26851_gb300 import build
    build.build()
    import paper_2510_26851_gb300 as j
    return j


@pytest.fixture(scope="module")
def box(J):
    spec = synth.BoxSpec("t", 200_000, 60.0, synth.linking_length(60.0, 200_000), 1200, 0.6, 23)
    pos, vel = synth.generate(spec, device="cuda")
    r = J.fof(pos, spec.L, spec.b, spec.min_size)
    J.sync()
    H = r.groups.n_halos
    pos_np, vel_np = pos.cpu().numpy(), vel.cpu().numpy()
    lab = oracle.fof_labels(pos_np, spec.L, spec.b)
    assert np.array_equal(r.label.cpu().numpy(), lab)
    hid, cnt = oracle.groups(lab, spec.min_size)
    return spec, pos, vel, r, H, pos_np, vel_np, hid


@pytest.mark.parametrize("fx,sv", [(0.5, 40.0), (0.8, 80.0), (0.5, np.inf), (1.0, 10.0)])
def test_sub_labels_bit_exact(J, box, fx, sv):
    spec, pos, vel, r, H, pos_np, vel_np, hid = box
    sx = (fx * spec.b) ** 2
    sv2 = sv ** 2 if np.isfinite(sv) else np.inf
    sub = J.subhalos(pos, vel, spec.L, r.groups, sx, sv2)
    J.sync()
    want = oracle.subhalo_labels(pos_np, vel_np, hid, H, spec.L, sx, sv2)
    assert np.array_equal(sub.cpu().numpy(), want)
    assert len(np.unique(want[hid >= 0])) >= H


def test_sub_halo_groups(J, box):
    spec, pos, vel, r, H, pos_np, vel_np, hid = box
    sx, sv = (0.5 * spec.b) ** 2, 40.0 ** 2
    sub = J.subhalos(pos, vel, spec.L, r.groups, sx, sv)
    g = J.groups(sub, min_size=10)
    J.sync()
    want = oracle.subhalo_labels(pos_np, vel_np, hid, H, spec.L, sx, sv)
    sid, scnt = oracle.groups(want, 10)
    assert g.n_halos == len(scnt) > 0
    assert np.array_equal(g.halo_id.cpu().numpy(), sid)


def test_one_large_halo_and_wrap(J):
    # 3000 members in one halo across the periodic faces: long rows, many unions
    rng = np.random.default_rng(4)
    L = 20.0
    core = (np.array([0.02, 19.97, 10.0]) + rng.normal(0, 0.08, (3000, 3)))
    vel = rng.normal(0, 30.0, (3000, 3))
    vel[:1500] += [150.0, 0.0, 0.0]
    pos_np = np.concatenate([core % L, rng.uniform(0, L, (20000, 3))]).astype(np.float32)
    vel_np = np.concatenate([vel, rng.normal(0, 300, (20000, 3))]).astype(np.float32)
    pos = torch.from_numpy(pos_np).cuda()
    velt = torch.from_numpy(vel_np).cuda()
    b = 0.2
    r = J.fof(pos, L, b, 20)
    J.sync()
    lab = oracle.fof_labels(pos_np, L, b)
    hid, cnt = oracle.groups(lab, 20)
    assert cnt.max() >= 2900
    sx, sv = 0.05 ** 2, 45.0 ** 2
    sub = J.subhalos(pos, velt, L, r.groups, sx, sv)
    J.sync()
    assert np.array_equal(sub.cpu().numpy(), oracle.subhalo_labels(pos_np, vel_np, hid, len(cnt), L, sx, sv))
    # positions shifted by L wrap back to the same groups
    shifted = pos.clone()
    shifted[:, 0] += L
    sub2 = J.subhalos(shifted, velt, L, r.groups, sx, sv, wrap=True)
    J.sync()
    assert torch.equal(sub2, sub)
