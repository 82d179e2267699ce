"""The allocation-free profile entry point, sc_pressure_profile_noalloc.

Some callers cannot allocate device memory when they need a profile (all
device memory handed to their own pool, or a region where cudaMalloc's
implicit synchronisation is not allowed).  For them the library offers a
variant whose only scratch is a fixed array inside the library.  This test
calls it through the C ABI twice in a row and checks each result against the
context-based sc_pressure_profile, the entry point it stands in for.  It lives
in a file of its own that pytest collects last."""
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


def test_noalloc_profile_matches_context_profile(B):
    import torch

    shape = (40, 36, 34)
    nA0, nB0 = S.droplet(shape[::-1], (20, 18, 17), 8.0, n_in=0.85, n_out=0.15, amplitude=1e-2)
    p = B.make_params(shape, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F64, tau=(1.0, 0.9), G=2.5,
                      G_self=(-0.4, 0.1))
    sim = B.Simulation(p, nA0, nB0)
    sim.step(6)
    nA, nB, _ = sim.moments(with_u=False)
    centre = (20.0, 18.0, 17.0)
    calls = [(B.SC_PROFILE_RADIAL, 60, 0.5), (B.SC_PROFILE_PLANAR_Z, 34, 1.0)]
    for kind, nbins, bw in calls:  # two calls in a row share the library's scratch array
        want = sim.profile(kind, centre, bw, nbins).cpu().numpy()
        out = torch.full((nbins * 6,), float("nan"), dtype=torch.float64, device="cuda")
        B.sc_pressure_profile_noalloc(p, nA, nB, kind, centre, bw, nbins, out)
        torch.cuda.synchronize()
        got = out.view(nbins, 6).cpu().numpy()
        np.testing.assert_array_equal(got[:, 5], want[:, 5])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    import torch

    p = B.make_params((8, 8, 8))
    n = torch.ones(512, dtype=torch.float64, device="cuda")
    out = torch.empty(6 * 5000, dtype=torch.float64, device="cuda")
    with pytest.raises(B.ScError) as e:
        B.sc_pressure_profile_noalloc(p, n, n, B.SC_PROFILE_RADIAL, (4.0, 4.0, 4.0), 0.5, 5000, out)
    assert e.value.status == B.SC_EINVAL
    assert "4096" in str(e.value)
