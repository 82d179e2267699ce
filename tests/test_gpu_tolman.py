"""Tolman length on the paper's couplings (section 4; Eq. self_p, Eq. sigma_c):
the trends the paper states for its curvature-coefficient results, on a smaller
sweep -- delta vanishes for symmetric couplings, changes sign with dG_AB and is
larger in magnitude for negative dG_AB; sigma_0 is smallest near the symmetric
case.  Everything numerical runs on the device (batch, profiles, sigma[R],
slab sigma_0, curvature fit)."""
import math

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


def couplings(dGAB, dGc=0.4):
    Gc = -math.e ** 2  # G_c c_s^2 = -e^2 / 3
    return dict(G=1.5, G_self=(Gc * (1.0 - dGc * (1.0 + dGAB)), Gc * (1.0 - dGc)))


def test_paper_tolman_trends(B):
    import torch

    from paper_2112_02574_gb300 import tolman

    steps, sides, ntot = 16384, (25, 31, 37, 41, 51), 2.0
    sets = (0.0, 0.88, -0.88)
    members, flats = [], {}
    for d in sets:
        kw = dict(lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F32, **couplings(d))
        slab = lambda shape: S.slab(shape, shape[0] / 2, n_rich=0.95 * ntot, n_poor=0.05 * ntot, amplitude=1e-3)
        fl = tolman.flat_densities((16, 16, 128), slab, kw, steps)
        flats[d] = fl
        for L in sides:
            for sign in (1, -1):
                inside = (fl["A_in"], fl["B_in"]) if sign > 0 else (fl["A_out"], fl["B_out"])
                outside = (fl["A_out"], fl["B_out"]) if sign > 0 else (fl["A_in"], fl["B_in"])
                f = S.droplet_ab((L, L, L), (L // 2,) * 3, L / 4.0, inside[0], outside[0], inside[1], outside[1])
                members.append({"L": L, "R": L / 4.0, "sign": sign, "params": kw, "fields": f, "tag": d})
    drops = tolman.sweep(members, steps)
    delta, s0 = {}, {}
    for d in sets:
        ds = [x for x in drops if x["tag"] == d]
        assert all(tolman.usable(x) for x in ds)
        sig0 = torch.tensor([flats[d]["sigma0"]], dtype=torch.float64, device="cuda")
        delta[d] = tolman.fit(ds, sig0)["delta"]
        s0[d] = flats[d]["sigma0"]
    assert abs(delta[0.0]) < 0.02
    assert delta[0.88] < -0.1 and delta[-0.88] > 0.1
    assert abs(delta[-0.88]) > abs(delta[0.88])
    assert s0[0.0] < s0[0.88] and s0[0.0] < s0[-0.88]
    # symmetric couplings: A-rich and B-rich droplets of one size are the same droplet (A <-> B)
    sym = [x for x in drops if x["tag"] == 0.0]
    for a, b in zip(sym[0::2], sym[1::2]):
        assert a["R_s"] == pytest.approx(b["R_s"], rel=1e-4)
        assert a["sigma_s"] == pytest.approx(b["sigma_s"], rel=1e-4)
