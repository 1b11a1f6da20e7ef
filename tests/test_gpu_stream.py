"""Streaming FoF over slabs of cell layers on the GPU (Sec. 2.2 streaming
mode; Sec. 2.3 union-find fusion): host positions, one slab subset at a time
on the device, equal to the in-memory path and to the oracle for any number
of slabs, including a 256^3 box forced into 4 slabs."""
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


def in_memory(J, pos, L, b, min_size=20):
    r = J.fof(pos.cuda(), L, b, min_size)
    J.sync()
    return r.label.cpu(), r.groups.halo_id.cpu(), r.groups.n_halos


def test_box_256cubed_in_four_slabs(J):
    spec = synth.BOX_256
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    hpos = pos.cpu()
    lab, hid, H = J.fof_stream(hpos, spec.L, spec.b, 4, spec.min_size)
    lab0, hid0, H0 = in_memory(J, pos, spec.L, spec.b, spec.min_size)
    assert torch.equal(lab, lab0) and torch.equal(hid, hid0) and H == H0
    want = oracle.fof_labels_mt(hpos.numpy(), spec.L, spec.b)
    assert np.array_equal(lab.numpy(), want)


@pytest.mark.parametrize("S", [1, 2, 3, 7])
def test_clustered_box_any_slab_count(J, S):
    spec = synth.BoxSpec("t", 300_000, 70.0, synth.linking_length(70.0, 300_000), 2000, 0.6, 31,
                         velocities=False)
    pos, _ = synth.generate(spec, device="cpu", velocities=False)
    lab, hid, H = J.fof_stream(pos, spec.L, spec.b, S, spec.min_size)
    want = oracle.fof_labels(pos.numpy(), spec.L, spec.b)
    hid_ref, cnt_ref = oracle.groups(want, spec.min_size)
    assert np.array_equal(lab.numpy(), want)
    assert np.array_equal(hid.numpy(), hid_ref) and H == len(cnt_ref)


def test_one_layer_slabs_and_periodic_faces(J):
    rng = np.random.default_rng(12)
    L, b = 10.0, 0.4
    q = rng.uniform(0, L, (20000, 3))
    q[:, 2] = np.where(rng.random(20000) < 0.5, rng.uniform(0, 0.6, 20000), rng.uniform(L - 0.6, L, 20000))
    pos = torch.from_numpy(q.astype(np.float32))
    n = oracle.max_cells_per_axis(L, b)
    want = oracle.fof_labels(pos.numpy(), L, b)
    for S in (2, 5, n):
        lab, _, _ = J.fof_stream(pos, L, b, S, 5, n_axis=n)
        assert np.array_equal(lab.numpy(), want), S


def test_single_rank_slab_path_on_the_gpu(J):
    spec = synth.BoxSpec("t", 200_000, 60.0, synth.linking_length(60.0, 200_000), 1200, 0.6, 5,
                         velocities=False)
    pos, _ = synth.generate(spec, device="cpu", velocities=False)
    g, lab, hid, H = J.fof_slabs(pos, spec.L, spec.b, spec.min_size)
    want = oracle.fof_labels(pos.numpy(), spec.L, spec.b)
    hid_ref, cnt_ref = oracle.groups(want, spec.min_size)
    assert torch.equal(g, torch.arange(spec.N))
    assert np.array_equal(lab.numpy(), want) and np.array_equal(hid.numpy(), hid_ref) and H == len(cnt_ref)


def test_stream_rejects_bad_arguments(J):
    pos = torch.rand(1000, 3) * 10
    with pytest.raises(J.JfofError):
        J.fof_stream(pos, 10.0, 0.4, 0, 20)  # no slabs
    bad = pos.clone()
    bad[3, 2] = 10.0  # z == L is outside [0, L)
    with pytest.raises(J.JfofError) as e:
        J.fof_stream(bad, 10.0, 0.4, 2, 20)
    assert e.value.code == J.JFOF_ERANGE
