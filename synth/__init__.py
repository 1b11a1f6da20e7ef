"""Seeded synthetic inputs: clustered periodic boxes that stand in for the
paper's fastPM particle boxes (500 Mpc/h, 64^3-512^3 particles, b = 0.2 of the
mean spacing; jFoF Sec. 2) and its 1024^3 slab run (Sec. 2.3).

This module holds no FoF arithmetic.  It produces positions (and velocities)
only; both the CUDA path and the oracle consume exactly the same float32 bytes.

Recipe (all in float64, rounded once to float32 at the end):
  1. n_halos centres, uniform in [0, L)^3.
  2. raw member counts from the truncated power law dN/dn ~ n^-1.9 on
     [20, 2000] by inverse CDF, rescaled with largest-remainder rounding so that
     halos hold round(frac * N) particles exactly (each halo keeps >= 1).
  3. NFW radii: r200 = (3 n / (4 pi 200 nbar))^(1/3), nbar = N / L^3,
     concentration c ~ U(5, 10), r_s = r200 / c; member radius r_s * x with
     mu(x) = u mu(c), mu(x) = ln(1+x) - x/(1+x), solved by bisection;
     isotropic directions (normalised Gaussian triples).
  4. the remaining particles uniform in the box; everything wrapped mod L in
     float64, rounded to float32, a value equal to L mapped to 0.
  5. velocities (optional): halo bulk ~ N(0, 300^2) per component, members
     bulk + N(0, sigma_h^2) with sigma_h = 100 (n_h / 1000)^(1/3), background
     N(0, 300^2).
  6. the particle order is a seeded random permutation (no free locality).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch


@dataclass(frozen=True)
class BoxSpec:
    name: str
    N: int
    L: float
    b: float  # absolute linking length, exactly representable in float32
    n_halos: int
    frac: float
    seed: int
    velocities: bool = True
    min_size: int = 20
    extra: dict = field(default_factory=dict, compare=False)


def linking_length(L: float, N: int) -> float:
    """b = 0.2 of the mean interparticle spacing (Eq. 1 with b = 0.2), rounded
    once to float32.  For N = m^3 the spacing is L/m exactly."""
    m = round(N ** (1.0 / 3.0))
    if m ** 3 == N:
        v = L / (5.0 * m)
    else:
        v = L / (5.0 * (N ** (1.0 / 3.0)))
    return float(torch.tensor(v, dtype=torch.float32).item())


def _spec(name, N, L, n_halos, frac, seed, velocities=True, **extra):
    return BoxSpec(name, N, float(L), linking_length(float(L), N), n_halos, frac, seed,
                   velocities, 20, extra)


# The five workloads: labels-only small box; 256^3; 1024^3; a batch of 64
# uneven boxes; the 128^3 differentiable-mode box.
SMALL_32 = _spec("fof_32cubed_L100", 32 ** 3, 100.0, 200, 0.50, 0, velocities=False)
BOX_256 = _spec("fof_256cubed_L250", 256 ** 3, 250.0, 100_000, 0.60, 0)
BOX_1024 = _spec("fof_1024cubed_L1000", 1024 ** 3, 1000.0, 5_000_000, 0.55, 0)
DIFF_128 = _spec("diff_128cubed_L200", 128 ** 3, 200.0, 12_500, 0.60, 0)


def batch_specs(n_boxes: int = 64, seed: int = 0) -> list[BoxSpec]:
    """64 independent boxes: N log-uniform in [32^3, 192^3], L ~ U(50, 400),
    b = 0.2 of each box's mean spacing, halos in proportion to N (100k per
    256^3) holding 60%, box k generated with seed k."""
    g = torch.Generator().manual_seed(1000 + seed)
    u = torch.rand(n_boxes, generator=g, dtype=torch.float64)
    w = torch.rand(n_boxes, generator=g, dtype=torch.float64)
    lo, hi = math.log(32 ** 3), math.log(192 ** 3)
    out = []
    for k in range(n_boxes):
        N = int(round(math.exp(lo + (hi - lo) * float(u[k]))))
        L = 50.0 + 350.0 * float(w[k])
        L = float(torch.tensor(L, dtype=torch.float32).item())
        nh = max(1, int(round(N * 100_000 / 256 ** 3)))
        out.append(_spec(f"batch{k}", N, L, nh, 0.60, k))
    return out


def _member_counts(n_halos: int, target: int, g, device) -> torch.Tensor:
    u = torch.rand(n_halos, generator=g, device=device, dtype=torch.float64)
    a, b = 20.0 ** -0.9, 2000.0 ** -0.9
    raw = ((b - a) * u + a) ** (-1.0 / 0.9)
    scaled = raw * (target / raw.sum())
    base = torch.floor(scaled)
    rem = scaled - base
    deficit = int(target - int(base.sum().item()))
    cnt = base.to(torch.int64)
    if deficit > 0:
        idx = torch.argsort(rem, descending=True, stable=True)[:deficit]
        cnt[idx] += 1
    # every halo keeps at least one member; take the excess from the largest
    zero = cnt < 1
    nz = int(zero.sum().item())
    if nz:
        cnt[zero] = 1
        order = torch.argsort(cnt, descending=True, stable=True)
        cnt[order[:nz]] -= 1
    return cnt


def _nfw_x(u: torch.Tensor, c: torch.Tensor, iters: int = 48) -> torch.Tensor:
    """Solve mu(x) = u mu(c) for x in [0, c] by bisection (float64)."""
    def mu(x):
        return torch.log1p(x) - x / (1.0 + x)
    target = u * mu(c)
    lo = torch.zeros_like(c)
    hi = c.clone()
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = mu(mid) < target
        lo = torch.where(below, mid, lo)
        hi = torch.where(below, hi, mid)
    return 0.5 * (lo + hi)


def generate(spec: BoxSpec, device="cpu", velocities: bool | None = None,
             chunk: int = 1 << 25):
    """Return (pos[N,3] float32, vel[N,3] float32 or None) on ``device``."""
    dev = torch.device(device)
    want_vel = spec.velocities if velocities is None else velocities
    g = torch.Generator(device=dev).manual_seed(int(spec.seed))
    N, L = spec.N, float(spec.L)
    f64 = torch.float64
    H = spec.n_halos
    M = int(round(spec.frac * N))
    centres = torch.rand(H, 3, generator=g, device=dev, dtype=f64) * L
    cnt = _member_counts(H, M, g, dev)
    nbar = N / L ** 3
    r200 = (3.0 * cnt.to(f64) / (4.0 * math.pi * 200.0 * nbar)) ** (1.0 / 3.0)
    conc = 5.0 + 5.0 * torch.rand(H, generator=g, device=dev, dtype=f64)
    rs = r200 / conc
    bulk = torch.randn(H, 3, generator=g, device=dev, dtype=f64) * 300.0
    sig_h = 100.0 * (cnt.to(f64) / 1000.0) ** (1.0 / 3.0)

    pos = torch.empty(N, 3, device=dev, dtype=torch.float32)
    vel = torch.empty(N, 3, device=dev, dtype=torch.float32) if want_vel else None
    hidx_all = torch.repeat_interleave(torch.arange(H, device=dev), cnt)

    def finish(p64: torch.Tensor) -> torch.Tensor:
        w = torch.remainder(p64, L)
        w32 = w.to(torch.float32)
        return torch.where(w32 >= L, torch.zeros_like(w32), w32)

    for s in range(0, M, chunk):
        e = min(M, s + chunk)
        hidx = hidx_all[s:e]
        u = torch.rand(e - s, generator=g, device=dev, dtype=f64)
        x = _nfw_x(u, conc[hidx])
        d = torch.randn(e - s, 3, generator=g, device=dev, dtype=f64)
        d = d / torch.linalg.vector_norm(d, dim=1, keepdim=True).clamp_min(1e-300)
        p = centres[hidx] + (rs[hidx] * x)[:, None] * d
        pos[s:e] = finish(p)
        if want_vel:
            v = bulk[hidx] + torch.randn(e - s, 3, generator=g, device=dev, dtype=f64) \
                * sig_h[hidx][:, None]
            vel[s:e] = v.to(torch.float32)
        del hidx, u, x, d, p
    del hidx_all
    for s in range(M, N, chunk):
        e = min(N, s + chunk)
        p = torch.rand(e - s, 3, generator=g, device=dev, dtype=f64) * L
        pos[s:e] = finish(p)
        if want_vel:
            vel[s:e] = (torch.randn(e - s, 3, generator=g, device=dev, dtype=f64)
                        * 300.0).to(torch.float32)
    perm = torch.randperm(N, generator=g, device=dev)
    pos = pos[perm]
    if want_vel:
        vel = vel[perm]
    del perm
    return pos, vel


def lattice(m: int, spacing: float, offset: float = 0.0):
    """m^3 particles on a cubic lattice of the given spacing (float32), box
    L = m * spacing; positions are offset + spacing * index (float64, rounded)."""
    idx = torch.arange(m, dtype=torch.float64)
    gz, gy, gx = torch.meshgrid(idx, idx, idx, indexing="ij")
    p = torch.stack([gx, gy, gz], dim=-1).reshape(-1, 3) * spacing + offset
    L = m * spacing
    p = torch.remainder(p, L)
    return p.to(torch.float32), float(torch.tensor(L, dtype=torch.float32).item())


def uniform(N: int, L: float, seed: int, device="cpu"):
    """N particles uniform in [0, L)^3, float32."""
    g = torch.Generator(device=device).manual_seed(int(seed))
    p = torch.rand(N, 3, generator=g, device=device, dtype=torch.float64) * L
    p32 = p.to(torch.float32)
    return torch.where(p32 >= L, torch.zeros_like(p32), p32)
