"""GPU parity for the REINFORCE topological mode (Sec. 3.2, Eqs. 6-8): the
candidate list, the device exponential and edge uniforms, per-sample labels
and halo counts (bit-exact), and the score-function gradient against the
FP64 oracle with identical draws."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-4  # normwise relative error of the FP32 gradient vs the FP64 oracle


@pytest.fixture(scope="module")
def J():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_26851_gb300 import build
    build.build()
    import paper_2510_26851_gb300 as j
    return j


def small_box(N=60_000, L=60.0, seed=3):
    spec = synth.BoxSpec("t", N, L, synth.linking_length(L, N), max(1, N * 12500 // 128 ** 3), 0.6, seed)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    return spec, pos


def r_cut_of(b):
    return float(np.float32(1.5 * np.float32(b)))


def test_exp_bitwise_host_equals_device(J):
    x = np.concatenate([np.linspace(-87.0, 87.0, 1 << 21, dtype=np.float32),
                        np.float32([0.0, -0.0, 1e-30, -1e-30, 90.0, -90.0, 87.0, -87.0])])
    rng = np.random.default_rng(0)
    x = np.concatenate([x, rng.uniform(-87, 87, 1 << 20).astype(np.float32)])
    y_dev = J.eval_exp(torch.from_numpy(x).cuda()).cpu().numpy()
    y_host = oracle.exp32_array(x)
    assert np.array_equal(y_dev.view(np.uint32), y_host.view(np.uint32))


def test_edge_uniforms_bitwise(J):
    rng = np.random.default_rng(1)
    n = 20000
    i = rng.integers(0, 1 << 30, n).astype(np.int32)
    j = rng.integers(0, 1 << 30, n).astype(np.int32)
    k = rng.integers(0, 256, n).astype(np.int32)
    seed = 0x1234567890ABCDEF
    u = J.eval_edge_uniform(seed, *(torch.from_numpy(a).cuda() for a in (i, j, k))).cpu().numpy()
    ref = np.array([oracle.edge_uniform(seed, int(a), int(b), int(c)) for a, b, c in zip(i, j, k)], np.float32)
    assert np.array_equal(u, ref)


@pytest.mark.parametrize("form", [0, 1])
def test_pairs_bit_exact(J, form):
    spec, pos = small_box()
    b = spec.b
    coef = J.prob_coef(b, form, alpha=5.0)
    assert np.float32(coef) == oracle.prob_coef(b, form, alpha=5.0)
    pr = J.pairs(pos, spec.L, b, r_cut_of(b), prob_form=form, coef=coef)
    J.sync()
    pi, pj, pd, pp = oracle.pairs(pos.cpu().numpy(), spec.L, b, r_cut_of(b), form, coef)
    assert pr.E == len(pi) and pr.E > 10000
    assert np.array_equal(pr.i.cpu().numpy(), pi) and np.array_equal(pr.j.cpu().numpy(), pj)
    assert np.array_equal(pr.d.cpu().numpy().view(np.uint32), pd.view(np.uint32))
    assert np.array_equal(pr.p.cpu().numpy().view(np.uint32), pp.view(np.uint32))


def oracle_pairs(pos, L, b, form=0, coef=None):
    """The oracle's candidate list, computed from the positions alone."""
    coef = oracle.prob_coef(b, form) if coef is None else coef
    return oracle.pairs(pos.cpu().numpy(), L, b, r_cut_of(b), form, coef)


def assert_same_pairs(pr, ref):
    pi, pj, pd, pp = ref
    assert pr.E == len(pi)
    assert np.array_equal(pr.i.cpu().numpy(), pi) and np.array_equal(pr.j.cpu().numpy(), pj)
    assert np.array_equal(pr.d.cpu().numpy().view(np.uint32), pd.view(np.uint32))
    assert np.array_equal(pr.p.cpu().numpy().view(np.uint32), pp.view(np.uint32))


def seeded_advantage(K, seed):
    """Advantages A_k with sum 0, drawn on the host (independent of the GPU)."""
    a = np.random.default_rng(seed).standard_normal(K)
    a -= a.mean()
    return a


def test_samples_and_halo_counts_bit_exact(J):
    spec, pos = small_box()
    pr = J.pairs(pos, spec.L, spec.b)
    J.sync()
    pi, pj, pd, pp = oracle_pairs(pos, spec.L, spec.b)
    assert_same_pairs(pr, (pi, pj, pd, pp))
    K, seed = 13, 42  # K not a multiple of 4 or of the sample chunk
    labels, nh = J.reinforce_sample(pr, K, seed, spec.min_size)
    J.sync()
    ref_l, ref_n = oracle.reinforce_sample(spec.N, pi, pj, pp, K, seed, spec.min_size)
    assert np.array_equal(labels.cpu().numpy(), ref_l)
    assert np.array_equal(nh.cpu().numpy(), ref_n)
    # samples differ from one another and from plain FoF
    assert len({tuple(r[:2000]) for r in ref_l}) > 1


@pytest.mark.parametrize("form", [0, 1])
def test_gradient_matches_fp64_oracle(J, form):
    spec, pos = small_box(N=30_000, L=48.0, seed=4)
    coef = J.prob_coef(spec.b, form, alpha=0.5)
    pr = J.pairs(pos, spec.L, spec.b, prob_form=form, coef=coef)
    J.sync()
    pi, pj, pd, pp = oracle_pairs(pos, spec.L, spec.b, form, coef)
    assert_same_pairs(pr, (pi, pj, pd, pp))
    K, seed = 64, 7
    adv = seeded_advantage(K, 100 + form)
    g = J.reinforce_grad(pos, pr, K, seed, torch.from_numpy(adv.astype(np.float32)).cuda())
    J.sync()
    ref = oracle.reinforce_grad(pos.cpu().numpy(), spec.L, pi, pj, pp, K, seed,
                                adv.astype(np.float32).astype(np.float64), form, coef)
    got = g.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert np.linalg.norm(ref) > 0 and err <= GRAD_RTOL, err


def test_dense_clump_pairs_and_gradient(J):
    # 2500 particles in a cube of side 0.8 b: every pair of the clump is a
    # candidate, so the per-i pair lists and the reverse adjacency hold
    # segments of every length up to 2499 (warp and block sorts alike)
    rng = np.random.default_rng(9)
    L = 30.0
    b = float(np.float32(0.3))
    clump = 15.0 + rng.uniform(0.0, 0.8 * b, (2500, 3))
    bg = rng.uniform(0.0, L, (8000, 3))
    pos_np = np.concatenate([clump, bg]).astype(np.float32)
    pos_np = pos_np[rng.permutation(len(pos_np))]
    pos = torch.from_numpy(pos_np).cuda()
    coef = J.prob_coef(b, 0)
    pr = J.pairs(pos, L, b, r_cut_of(b), prob_form=0, coef=coef)
    J.sync()
    pi, pj, pd, pp = oracle.pairs(pos_np, L, b, r_cut_of(b), 0, coef)
    assert pr.E == len(pi) and pr.E > 2500 * 2499 // 2
    assert np.array_equal(pr.i.cpu().numpy(), pi) and np.array_equal(pr.j.cpu().numpy(), pj)
    assert np.array_equal(pr.p.cpu().numpy().view(np.uint32), pp.view(np.uint32))
    K, seed = 8, 3
    adv = seeded_advantage(K, 9).astype(np.float32)
    g = J.reinforce_grad(pos, pr, K, seed, torch.from_numpy(adv).cuda())
    J.sync()
    ref = oracle.reinforce_grad(pos_np, L, pi, pj, pp, K, seed, adv.astype(np.float64), 0, coef)
    got = g.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert np.linalg.norm(ref) > 0 and err <= GRAD_RTOL, err


def test_autograd_function(J):
    spec, pos = small_box(N=20_000, L=42.0, seed=5)
    pr = J.pairs(pos, spec.L, spec.b)
    K, seed = 32, 11
    _, nh = J.reinforce_sample(pr, K, seed, 5)
    losses = nh.float()
    x = pos.clone().requires_grad_(True)
    out = J.ReinforceFoF.apply(x, pr, losses, seed)
    out.backward()
    g = J.reinforce_grad(pos, pr, K, seed, (losses - losses.mean()).contiguous())
    J.sync()
    assert torch.equal(x.grad, g)
    assert abs(out.item() - losses.mean().item()) < 1e-6


def test_diff_box_128cubed_full_size(J):
    # the 128^3 differentiable-mode box (K = 256): the full pair list
    # bit-exact against the oracle's own list; 16 of the 256 samples (labels
    # and halo counts) bit-exact, the oracle fed only its own list; the
    # gradient on a sampled particle subset with host-drawn advantages
    spec = synth.DIFF_128
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    pos_np = pos.cpu().numpy()
    pr = J.pairs(pos, spec.L, spec.b)
    J.sync()
    pi, pj, pd, pp = oracle_pairs(pos, spec.L, spec.b)
    assert_same_pairs(pr, (pi, pj, pd, pp))
    K, seed = 256, 0
    labels, nh = J.reinforce_sample(pr, K, seed, spec.min_size)
    J.sync()
    ks = [0, 1, 2, 3, 5, 17, 64, 100, 127, 128, 129, 200, 211, 233, 254, 255]
    with ThreadPoolExecutor(max_workers=min(len(ks), os.cpu_count() or 1)) as ex:
        refs = list(ex.map(lambda k: oracle.reinforce_sample_one(spec.N, pi, pj, pp, k, seed, spec.min_size), ks))
    for k, (lab, h) in zip(ks, refs):
        assert np.array_equal(labels[k].cpu().numpy(), lab), k
        assert nh[k].item() == h
    adv = seeded_advantage(K, 128).astype(np.float32)
    g = J.reinforce_grad(pos, pr, K, seed, torch.from_numpy(adv).cuda()).cpu().numpy().astype(np.float64)
    mask = np.zeros(spec.N, np.uint8)
    mask[np.random.default_rng(2).choice(spec.N, 3000, replace=False)] = 1
    ref = oracle.reinforce_grad_masked(pos_np, spec.L, pi, pj, pp, K, seed, adv.astype(np.float64), 0,
                                       J.prob_coef(spec.b, 0), mask)
    sel = mask.astype(bool)
    err = np.linalg.norm(g[sel] - ref[sel]) / np.linalg.norm(ref[sel])
    assert err <= GRAD_RTOL, err
