"""GPU parity for the batched form: many independent boxes of uneven size in
one CUDA-graph launch give, box by box, the oracle's labels, halo ids and
halo counts; the per-box loop gives the same; graph replays are stable; the
autotuner's choice leaves labels unchanged."""
from concurrent.futures import ThreadPoolExecutor

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


def make_batch(specs):
    pos = []
    for sp in specs:
        p, _ = synth.generate(sp, device="cuda", velocities=False)
        pos.append(p)
    off = np.concatenate([[0], np.cumsum([sp.N for sp in specs])]).astype(np.int64)
    return torch.cat(pos).contiguous(), off


def check_box(J, pos_np, sp, lab, hid, nh):
    ref = oracle.fof_labels(pos_np, sp.L, sp.b)
    assert np.array_equal(lab, ref), sp.name
    hid_ref, cnt_ref = oracle.groups(ref, sp.min_size)
    assert np.array_equal(hid, hid_ref), sp.name
    assert nh == len(cnt_ref), sp.name


def test_small_batch_graph_and_loop_match_oracle(J):
    rng = np.random.default_rng(0)
    specs = []
    for k, N in enumerate([700, 5000, 33, 20000, 1, 64000, 9000, 1500]):
        L = float(np.float32(rng.uniform(20, 80)))
        specs.append(synth.BoxSpec(f"b{k}", N, L, synth.linking_length(L, N), max(1, N // 300), 0.6, k,
                                   velocities=False))
    pos, off = make_batch(specs)
    bt = J.Batch(off, [s.L for s in specs], [s.b for s in specs], min_size=20)
    outs = []
    for use_graph in (True, True, False):
        lab, hid, nh = bt.run(pos, use_graph=use_graph)
        J.sync()
        outs.append((lab.cpu().numpy().copy(), hid.cpu().numpy().copy(), nh.cpu().numpy().copy()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
    lab, hid, nh = outs[0]
    pos_np = pos.cpu().numpy()
    for k, sp in enumerate(specs):
        s, e = off[k], off[k + 1]
        check_box(J, pos_np[s:e], sp, lab[s:e], hid[s:e], nh[k])


def test_batch_of_64_uneven_boxes(J):
    specs = synth.batch_specs()
    pos, off = make_batch(specs)
    assert 2e7 < off[-1] < 3e8
    bt = J.Batch(off, [s.L for s in specs], [s.b for s in specs], min_size=20)
    lab_g, hid_g, nh_g = [t.cpu().numpy().copy() for t in bt.run(pos, use_graph=True)]
    J.sync()
    lab_l, hid_l, nh_l = [t.cpu().numpy().copy() for t in bt.run(pos, use_graph=False)]
    J.sync()
    assert np.array_equal(lab_g, lab_l) and np.array_equal(hid_g, hid_l) and np.array_equal(nh_g, nh_l)
    # every box against the oracle (boxes on parallel host threads)
    pos_np = pos.cpu().numpy()

    def one(k):
        s, e = off[k], off[k + 1]
        check_box(J, pos_np[s:e], specs[k], lab_g[s:e], hid_g[s:e], nh_g[k])

    with ThreadPoolExecutor(max_workers=oracle.default_threads()) as ex:
        list(ex.map(one, range(len(specs))))


def test_autotuner_choice_keeps_labels(J):
    spec = synth.BoxSpec("t", 400_000, 73.0, synth.linking_length(73.0, 400_000), 2400, 0.6, 12,
                         velocities=False)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    n, S, T, W, ms = J.autotune(pos, spec.L, spec.b, spec.min_size)
    assert ms > 0 and n >= 3 and W in (0, 1, 2)
    # the same size bucket: the kept choice comes back without timing
    assert J.autotune(pos, spec.L, spec.b, spec.min_size, use_cache=True) == (n, S, T, W, ms)
    ref = oracle.fof_labels(pos.cpu().numpy(), spec.L, spec.b)
    try:
        J.set_cell_classes(S, T)
        J.set_cta_shape(W)
        r = J.fof(pos, spec.L, spec.b, spec.min_size, n_axis=n)
        J.sync()
    finally:
        J.set_cell_classes()
        J.set_cta_shape(0)
    assert np.array_equal(r.label.cpu().numpy(), ref)


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_labels_do_not_depend_on_the_cta_shape(J, shape):
    # every CTA shape of the four list-driven link kernels, with many dense
    # and medium cells (a low dense threshold)
    spec = synth.BoxSpec("t", 300_000, 50.0, synth.linking_length(50.0, 300_000), 2500, 0.7, 14,
                         velocities=False)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    ref = oracle.fof_labels(pos.cpu().numpy(), spec.L, spec.b)
    try:
        J.set_cta_shape(shape)
        for S, T in ((8, 96), (4, 32)):
            J.set_cell_classes(S, T)
            r = J.fof(pos, spec.L, spec.b, spec.min_size)
            J.sync()
            assert np.array_equal(r.label.cpu().numpy(), ref), (shape, S, T)
    finally:
        J.set_cell_classes()
        J.set_cta_shape(0)


def test_tuned_batch_matches_oracle(J):
    rng = np.random.default_rng(5)
    specs = []
    for k, N in enumerate([40_000, 90_000, 40_000, 250_000, 7_000, 90_000]):
        L = float(np.float32(rng.uniform(40, 90)))
        specs.append(synth.BoxSpec(f"u{k}", N, L, synth.linking_length(L, N), max(1, N // 200), 0.6, 40 + k,
                                   velocities=False))
    pos, off = make_batch(specs)
    pos_np = pos.cpu().numpy()
    bt, picks = J.Batch.tuned(pos, off, [s.L for s in specs], [s.b for s in specs], min_size=20, reps=1)
    bt2, picks2, ms = J.tune_batch(pos, off, [s.L for s in specs], [s.b for s in specs], min_size=20, reps=1)
    assert len(picks) == len(picks2) == len(specs) and ms > 0
    for b_ in (bt, bt2):
        lab, hid, nh = [t.cpu().numpy().copy() for t in b_.run(pos, use_graph=True)]
        J.sync()
        for k, sp in enumerate(specs):
            s, e = off[k], off[k + 1]
            check_box(J, pos_np[s:e], sp, lab[s:e], hid[s:e], nh[k])
