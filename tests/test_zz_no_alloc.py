"""The no-allocation entry point jfof_fof_static against jfof_fof, through
the C ABI, on two calls in a row.

jfof_fof_static runs the same pipeline on a fixed device array owned by the
library instead of a caller workspace.  It serves callers that must not
allocate device memory: an analysis hook inside a simulation or framework
that owns all device memory through its own pool, or a latency-critical path
that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
impose.  Consecutive calls use different boxes, so each reuses the shared
scratch left by the one before.  This file is collected last on purpose."""
import ctypes

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


def outputs(r):
    g = r.groups
    H = g.n_halos
    M = int(g.halo_start[H].item())
    return (r.label.cpu().numpy(), g.halo_id.cpu().numpy(), g.count[:H].cpu().numpy(),
            g.halo_start[:H + 1].cpu().numpy(), g.members[:M].cpu().numpy(), H)


def test_static_scratch_matches_workspace_path_twice(J):
    # boxes in a row, large then small then large again: the smaller call's
    # layout lies inside bytes the larger one left behind, so stale scratch
    # would show; each result must equal jfof_fof and the oracle
    big = synth.BoxSpec("s2", 100_000, 70.0, synth.linking_length(70.0, 100_000), 700, 0.5, 22,
                        velocities=False)
    small = synth.BoxSpec("s1", 60_000, 50.0, synth.linking_length(50.0, 60_000), 400, 0.6, 21,
                          velocities=False)
    for spec in (big, small, big):
        pos, _ = synth.generate(spec, device="cuda", velocities=False)
        got = J.fof_static(pos, spec.L, spec.b, spec.min_size)
        J.sync()
        want = J.fof(pos, spec.L, spec.b, spec.min_size)
        J.sync()
        a, b = outputs(got), outputs(want)
        assert a[5] == b[5] and a[5] > 10
        for x, y in zip(a[:5], b[:5]):
            assert np.array_equal(x, y)
        lab_ref = oracle.fof_labels(pos.cpu().numpy(), spec.L, spec.b)
        hid_ref, cnt_ref = oracle.groups(lab_ref, spec.min_size)
        assert np.array_equal(a[0], lab_ref)
        assert np.array_equal(a[1], hid_ref) and np.array_equal(a[2], cnt_ref)


def test_static_scratch_rejects_inputs_beyond_its_limit(J):
    N = 1_000_000
    pos = torch.zeros(N, 3, device="cuda")
    with pytest.raises(J.JfofError) as e:
        J.fof_static(pos, 100.0, 0.2)
    assert e.value.code == J.JFOF_ENOMEM
    J.sync()
