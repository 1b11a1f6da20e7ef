"""Slabs of cell layers (Sec. 2.2 streaming mode, Sec. 2.3 slab decomposition
with union-find fusion), host side, no GPU: the library's slab selection and
union-find fusion, with the oracle linking each slab's subset, must give the
oracle's labels of the whole box; the same path over two gloo ranks."""
import os
import queue
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def J():
    from paper_2510_26851_gb300 import build
    build.build()
    import paper_2510_26851_gb300 as j
    return j


def layers(pos, L, n):
    # the z cell layer, in binary32 as the library computes it
    u = pos[:, 2].astype(np.float32) * np.float32(n / L)
    return np.clip(np.floor(u).astype(np.int64), 0, n - 1)


def oracle_link(pos_s, L, b, n):
    # the oracle links one slab's subset in the full periodic box
    return torch.from_numpy(oracle.fof_labels(pos_s.numpy(), L, b, n_axis=n))


def clustered(N=20000, L=40.0, seed=4, boost=1.5):
    spec = synth.BoxSpec("t", N, L, synth.linking_length(L, N) * boost, N // 150, 0.6, seed)
    pos, _ = synth.generate(spec, velocities=False)
    return spec, pos


def test_slab_select_layers_and_core_partition(J):
    spec, pos = clustered()
    n = J.default_cells_per_axis(spec.N, spec.L, spec.b)
    lay = layers(pos.numpy(), spec.L, n)
    for S in (1, 2, 3, 5, n):
        owner = np.full(spec.N, -1)
        for s in range(S):
            idx, core = J.slab_select(pos, spec.L, spec.b, S, s)
            idx, core = idx.numpy(), core.numpy().astype(bool)
            assert np.all(np.diff(idx) > 0)
            z0, z1 = n * s // S, n * (s + 1) // S
            span = z1 - z0 + 2
            want = np.nonzero(((lay - (z0 - 1)) % n < span) if span < n else np.ones(spec.N, bool))[0]
            assert np.array_equal(idx, want), (S, s)
            assert np.array_equal(core, (lay[idx] >= z0) & (lay[idx] < z1))
            assert np.all(owner[idx[core]] == -1)
            owner[idx[core]] = s
        assert np.all(owner >= 0), S


def test_merge_labels_hand_cases(J):
    i32 = lambda v: torch.tensor(v, dtype=torch.int32)
    # 0-1 joined, 3-5 joined via pre, 5-2 joined: classes {0,1}, {2,3,5}, {4}
    pre = i32([0, 0, 2, 5, 4, 5])
    out = J.merge_labels(pre, i32([1, 5]), i32([0, 2]))
    assert out.tolist() == [0, 0, 2, 2, 4, 2]
    assert J.merge_labels(pre, i32([]), i32([])).tolist() == [0, 0, 2, 5, 4, 5]
    with pytest.raises(J.JfofError):
        J.merge_labels(i32([0, 7]), i32([]), i32([]))


def emulate_stream(J, pos, L, b, S, n=0):
    # the streaming path with the oracle as the per-slab linker
    N = pos.shape[0]
    n = n or J.default_cells_per_axis(N, L, b)
    pre = torch.arange(N, dtype=torch.int32)
    a, c = [], []
    for s in range(S):
        idx, core = J.slab_select(pos, L, b, S, s, n_axis=n)
        if idx.numel() == 0:
            continue
        lab = oracle_link(pos[idx].contiguous(), L, b, n).long()
        R = idx[lab]
        k = core.bool()
        pre[idx[k]] = R[k].to(torch.int32)
        a.append(idx[~k])
        c.append(R[~k])
    g = torch.cat(a)
    return J.merge_labels(pre, pre[g].contiguous(), torch.cat(c).to(torch.int32).contiguous())


@pytest.mark.parametrize("S", [1, 2, 3, 4, 7])
def test_slab_fusion_equals_whole_box(J, S):
    spec, pos = clustered()
    want = oracle.fof_labels(pos.numpy(), spec.L, spec.b)
    assert len(set(want.tolist())) < spec.N - 1000
    got = emulate_stream(J, pos, spec.L, spec.b, S)
    assert np.array_equal(got.numpy(), want)


def test_slab_fusion_one_layer_slabs_and_periodic_faces(J):
    # groups straddling the z = 0 / L faces and slabs of a single layer
    rng = np.random.default_rng(8)
    L, b = 10.0, 0.4
    q = rng.uniform(0, L, (5000, 3))
    q[:, 2] = np.where(rng.random(5000) < 0.5, rng.uniform(0, 0.6, 5000), rng.uniform(L - 0.6, L, 5000))
    pos = torch.from_numpy(q.astype(np.float32))
    n = oracle.max_cells_per_axis(L, b)
    want = oracle.fof_brute(pos.numpy(), L, b)
    for S in (2, 3, n):
        assert np.array_equal(emulate_stream(J, pos, L, b, S, n=n).numpy(), want), S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2510_26851_gb300 as J
        spec, pos = clustered()
        g, lab, hid, H = J.fof_slabs(pos, spec.L, spec.b, 20, link_slab=oracle_link)
        q.put((rank, g.numpy(), lab.numpy(), hid.numpy(), H))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_fof_slabs_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in range(world):
            res.append(q.get(timeout=240))
    except queue.Empty:
        pass
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert len(res) == world and all(p.exitcode == 0 for p in procs)
    spec, pos = clustered()
    want = oracle.fof_labels(pos.numpy(), spec.L, spec.b)
    hid_ref, cnt_ref = oracle.groups(want, 20)
    seen = np.zeros(spec.N, bool)
    for rank, g, lab, hid, H in res:
        assert not seen[g].any()
        seen[g] = True
        assert np.array_equal(lab, want[g]), rank
        assert np.array_equal(hid, hid_ref[g]), rank
        assert H == len(cnt_ref)
    assert seen.all()
