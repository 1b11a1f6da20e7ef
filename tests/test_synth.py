"""The synthetic input recipe (no GPU): the clustered-box generator holds no
FoF arithmetic, so these pin only what it promises -- exact linking lengths,
seeded determinism, positions in [0, L), member counts that sum exactly to the
halo fraction, NFW radii that solve their equation, velocity dispersions, and
the 64-box batch's ranges."""
import math

import numpy as np
import torch

import synth


def test_linking_length_is_exact_for_cubes():
    # 0.2 of the mean spacing L/m, rounded once to float32
    assert synth.linking_length(1000.0, 1024 ** 3) == 0.1953125
    assert synth.linking_length(250.0, 256 ** 3) == 0.1953125
    assert synth.linking_length(100.0, 32 ** 3) == 0.625
    assert synth.linking_length(200.0, 128 ** 3) == 0.3125
    b = synth.linking_length(129.0, 73228)
    assert b == float(np.float32(129.0 / (5.0 * 73228 ** (1 / 3))))


def test_generation_is_seeded_and_inside_the_box():
    spec = synth.BoxSpec("t", 20_000, 40.0, synth.linking_length(40.0, 20_000), 100, 0.5, 3)
    p1, v1 = synth.generate(spec)
    p2, v2 = synth.generate(spec)
    assert torch.equal(p1, p2) and torch.equal(v1, v2)
    other = synth.BoxSpec("t", 20_000, 40.0, spec.b, 100, 0.5, 4)
    assert not torch.equal(synth.generate(other)[0], p1)
    assert p1.dtype == torch.float32 and tuple(p1.shape) == (20_000, 3)
    assert bool((p1 >= 0).all()) and bool((p1 < 40.0).all())
    assert synth.generate(spec, velocities=False)[1] is None


def test_member_counts_sum_to_the_halo_fraction():
    g = torch.Generator().manual_seed(0)
    for H, M in ((200, 16_384), (100_000, 10_066_330), (7, 50)):
        cnt = synth._member_counts(H, M, g, "cpu")
        assert int(cnt.sum()) == M and bool((cnt >= 1).all()) and cnt.shape[0] == H
    # the raw draw is a truncated power law on [20, 2000] with mean ~107: the
    # rescaled counts of a large draw keep that shape
    cnt = synth._member_counts(200_000, int(round(107.0 * 200_000)), g, "cpu").double()
    assert 15 <= float(cnt.min()) and float(cnt.max()) <= 2100
    assert abs(float(cnt.mean()) - 107.0) < 1.0


def test_nfw_radii_solve_the_mass_profile():
    # x solves mu(x) = u mu(c), mu(x) = ln(1 + x) - x / (1 + x)
    u = torch.tensor([0.0, 0.1, 0.5, 0.9, 1.0], dtype=torch.float64)
    c = torch.tensor([5.0, 7.0, 10.0, 6.0, 8.0], dtype=torch.float64)
    x = synth._nfw_x(u, c)
    mu = lambda t: torch.log1p(t) - t / (1.0 + t)
    assert torch.allclose(mu(x), u * mu(c), rtol=0, atol=1e-12)
    assert bool((x >= 0).all()) and bool((x <= c).all())


def test_velocity_dispersions():
    # background: N(0, 300^2) per component; halo members: bulk + sigma_h
    spec = synth.BoxSpec("t", 200_000, 100.0, synth.linking_length(100.0, 200_000), 10, 0.05, 5)
    _, v = synth.generate(spec)
    assert v.dtype == torch.float32 and tuple(v.shape) == (200_000, 3)
    # 95% of particles are background, so the overall spread is close to 300
    s = float(v.double().std())
    assert 280.0 < s < 320.0


def test_batch_specs_ranges():
    specs = synth.batch_specs()
    assert len(specs) == 64
    assert [s.seed for s in specs] == list(range(64))
    for s in specs:
        assert 32 ** 3 <= s.N <= 192 ** 3
        assert 50.0 <= s.L <= 400.0
        assert s.b == synth.linking_length(s.L, s.N)
        assert s.frac == 0.6 and s.min_size == 20
        assert s.n_halos == max(1, int(round(s.N * 100_000 / 256 ** 3)))
    logs = np.log([s.N for s in specs])
    assert logs.min() < math.log(64 ** 3) and logs.max() > math.log(128 ** 3)  # spread over the range
