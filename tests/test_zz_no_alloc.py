"""The allocation-free profile entry point, sc_pressure_profile_noalloc.

Some callers cannot allocate device memory when they need a profile (all
device memory handed to their own pool, or a region where cudaMalloc's
implicit synchronisation is not allowed).  For them the library offers a
variant whose only scratch is a fixed array inside the library.  These tests
call it through the C ABI, two calls in a row for each model, and check each
result against the context-based sc_pressure_profile, the entry point it stands
in for, at the profile tolerance of the parity tests (rtol 1e-12, exact counts).
The file is collected last."""
import numpy as np
import pytest

import sc_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2112_02574_gb300 import binding

    return binding


def _noalloc(B, p, nA, nB, kind, centre, bw, nbins):
    import torch

    out = torch.full((nbins * 6,), float("nan"), dtype=torch.float64, device="cuda")
    B.sc_pressure_profile_noalloc(p, nA, nB, kind, centre, bw, nbins, out)
    torch.cuda.synchronize()
    return out.view(nbins, 6).cpu().numpy()


MODELS = [  # (lattice, stencil, psi_self)
    (0, 0, 1), (0, 0, 0), (1, 0, 1), (1, 0, 0), (1, 1, 1), (1, 1, 0),
]


@pytest.mark.parametrize("lattice,stencil,psi", MODELS)
def test_noalloc_profile_matches_context_profile(B, lattice, stencil, psi):
    shape = (40, 36, 34) if lattice == 1 else (64, 60, 1)
    centre = (20.0, 18.0, 17.0) if lattice == 1 else (32.0, 30.0, 0.0)
    nA0, nB0 = S.droplet(shape[::-1], tuple(int(c) for c in centre), 8.0, n_in=0.85, n_out=0.15, amplitude=1e-2)
    p = B.make_params(shape, lattice=lattice, stencil=stencil, psi_self=psi, storage=B.SC_STORE_F64,
                      tau=(1.0, 0.9), G=2.5, G_self=(-0.4, 0.1))
    sim = B.Simulation(p, nA0, nB0)
    sim.step(6)
    nA, nB, _ = sim.moments(with_u=False)
    calls = [(B.SC_PROFILE_RADIAL, 60, 0.5), (B.SC_PROFILE_PLANAR_Z, shape[2], 1.0), (B.SC_PROFILE_AXIS_X, 20, 1.0)]
    for kind, nbins, bw in calls:  # calls in a row share the library's scratch array
        want = sim.profile(kind, centre, bw, nbins).cpu().numpy()
        got = _noalloc(B, p, nA, nB, kind, centre, bw, nbins)
        np.testing.assert_array_equal(got[:, 5], want[:, 5])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_noalloc_profile_at_its_bin_limit(B):
    """nbins = 4096, the largest request the fixed scratch takes (192 KiB of shared bins per block,
    21 partial blocks): radial shells of 0.0085 lattice units on a 40^3 lattice fill bins up to
    r = 34.6, then a second call with few bins reuses the same scratch."""
    shape = (40, 40, 40)
    nA0, nB0 = S.droplet(shape[::-1], (20, 20, 20), 9.0, n_in=0.85, n_out=0.15, amplitude=1e-2)
    p = B.make_params(shape, psi_self=1, storage=B.SC_STORE_F64, G=2.5, G_self=(-0.4, 0.0))
    sim = B.Simulation(p, nA0, nB0)
    sim.step(3)
    nA, nB, _ = sim.moments(with_u=False)
    for nbins, bw in ((4096, 0.0085), (7, 0.5)):
        want = sim.profile(B.SC_PROFILE_RADIAL, (20.0, 20.0, 20.0), bw, nbins).cpu().numpy()
        got = _noalloc(B, p, nA, nB, B.SC_PROFILE_RADIAL, (20.0, 20.0, 20.0), bw, nbins)
        np.testing.assert_array_equal(got[:, 5], want[:, 5])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
        if nbins == 4096:
            assert got[:, 5].sum() == 40**3 and (got[4000:, 5] > 0).any()


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    import torch

    p = B.make_params((8, 8, 8))
    n = torch.ones(512, dtype=torch.float64, device="cuda")
    out = torch.empty(6 * 5000, dtype=torch.float64, device="cuda")
    with pytest.raises(B.ScError) as e:
        B.sc_pressure_profile_noalloc(p, n, n, B.SC_PROFILE_RADIAL, (4.0, 4.0, 4.0), 0.5, 5000, out)
    assert e.value.status == B.SC_EINVAL
    assert "4096" in str(e.value)
