"""GPU parity for the decorated frozen assignment and the soft mass function
(Sec. 3.1.1, Eq. 5): the decoration (particle standard deviation about each
halo centre) and the soft histogram of log-masses against the FP64 oracle,
and the gradient to the positions (histogram VJP, g_D = -kappa g_ell / D,
decoration adjoint) against the oracle's chain of the same adjoints."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DSIG_RTOL = 1e-5   # compensated binary32 sums about a binary32 centre
GRAD_RTOL = 1e-4   # normwise, as the other adjoints


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
    spec = synth.BoxSpec("t", 200_000, 60.0, synth.linking_length(60.0, 200_000), 1200, 0.6, 17,
                         velocities=False)
    pos, _ = synth.generate(spec, device="cuda", velocities=False)
    r = J.fof(pos, spec.L, spec.b, spec.min_size)
    J.sync()
    H = r.groups.n_halos
    pos_np = pos.cpu().numpy()
    lab_ref = oracle.fof_labels(pos_np, spec.L, spec.b)
    assert np.array_equal(r.label.cpu().numpy(), lab_ref)
    hid_ref, cnt_ref = oracle.groups(lab_ref, spec.min_size)
    assert H == len(cnt_ref) > 100
    _, com_ref, _, _ = oracle.halo_props(pos_np.astype(np.float64), np.zeros((spec.N, 3)), hid_ref, H, spec.L)
    D_ref = oracle.halo_decoration(pos_np.astype(np.float64), hid_ref, H, spec.L, com_ref)
    return spec, pos, r, H, hid_ref, cnt_ref, com_ref, D_ref


def edges_for(cnt):
    lo, hi = np.log(20.0) - 0.2, np.log(cnt.max()) + 0.5
    return np.linspace(lo, hi, 13).astype(np.float32)


def test_decoration_matches_fp64_oracle(J, box):
    spec, pos, r, H, hid_ref, cnt_ref, com_ref, D_ref = box
    p = J.halo_props(pos, None, spec.L, r.groups)
    D = J.halo_decoration(pos, spec.L, r.groups, p.com)
    J.sync()
    got = D[:H].cpu().numpy().astype(np.float64)
    assert (np.abs(got - D_ref) <= DSIG_RTOL * D_ref).all(), np.max(np.abs(got - D_ref) / D_ref)


def test_soft_hmf_and_gradient_match_oracle(J, box):
    spec, pos, r, H, hid_ref, cnt_ref, com_ref, D_ref = box
    edges = edges_for(cnt_ref)
    width, kappa = 0.15, 1.3
    e_dev = torch.from_numpy(edges).cuda()
    hist = J.soft_hmf(r.groups, e_dev, width)
    J.sync()
    ell = np.log(cnt_ref.astype(np.float64))
    want = oracle.soft_hist(ell, edges.astype(np.float64), width)
    got = hist.cpu().numpy().astype(np.float64)
    assert (np.abs(got - want) <= 1e-5 * np.maximum(1.0, np.abs(want)) + 1e-6 * H).all(), (got, want)
    # gradient of sum_k w_k hist_k to the positions
    w = np.random.default_rng(2).normal(size=len(edges) - 1)
    x = pos.clone().requires_grad_(True)
    out = J.DecoratedHMF.apply(x, r.groups, spec.L, e_dev, width, kappa)
    (out * torch.from_numpy(w.astype(np.float32)).cuda()).sum().backward()
    J.sync()
    assert torch.equal(out.detach(), hist)
    g_ell = oracle.soft_hist_backward(ell, edges.astype(np.float64), width, w)
    ref = oracle.halo_decoration_backward(pos.detach().cpu().numpy().astype(np.float64), hid_ref, H, spec.L,
                                          com_ref, D_ref, -kappa * g_ell / D_ref)
    g = x.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert np.linalg.norm(ref) > 0 and err <= GRAD_RTOL, err
    assert not g[hid_ref < 0].any()


def test_soft_hmf_is_deterministic_and_hard_in_the_limit(J, box):
    spec, pos, r, H, hid_ref, cnt_ref, com_ref, D_ref = box
    edges = np.log(np.array([17.5, 30.5, 60.5, 120.5, 1e6])).astype(np.float32)  # no log-count on an edge
    e_dev = torch.from_numpy(edges).cuda()
    h1 = J.soft_hmf(r.groups, e_dev, 1e-4)
    h2 = J.soft_hmf(r.groups, e_dev, 1e-4)
    J.sync()
    assert torch.equal(h1, h2)
    hard, _ = np.histogram(cnt_ref, bins=np.exp(edges.astype(np.float64)))
    assert np.allclose(h1.cpu().numpy(), hard, atol=1e-3)
