"""Section 4's convergence and acceptance measures and the retirement of
converged members from a batch:

* the velocity criterion dU = (1/N) sum_x sum_alpha |u(t) - u(t0)| and the
  centre of mass of a component's density excess, from the FP64 path, against
  the same quantities from the FP64 oracle's fields;
* a retired batch member keeps the state it had when it retired (equal, bit for
  bit, to a lone run of that many steps) while the others go on."""
import numpy as np
import pytest

import oracle
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


def test_velocity_change_and_centre_of_mass_match_oracle(B):
    shape = (40, 36, 34)
    nA0, nB0 = S.droplet(shape[::-1], (21, 17, 16), 7.0, n_in=0.85, n_out=0.15, amplitude=1e-2)
    kw = dict(G=2.5, G_self=(-0.4, 0.1), tau=(1.0, 0.9))
    sim = B.Simulation(B.make_params(shape, psi_self=1, storage=B.SC_STORE_F64, **kw), nA0, nB0)
    op = oracle.Params(shape=shape, lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, **kw)
    f = oracle.init(op, nA0, nB0)
    sim.step(3)
    f = oracle.step(op, f, 3)
    _, _, u_prev = sim.moments()
    u_prev = u_prev.clone()
    _, _, u3 = oracle.moments(op, f)
    sim.step(5)
    f = oracle.step(op, f, 5)
    a8, b8, u8 = oracle.moments(op, f)
    du = sim.velocity_change(u_prev).item()
    want = np.abs(u8 - u3).sum() / a8.size
    assert want > 1e-6
    assert du == pytest.approx(want, rel=1e-10)
    # u_prev now holds the velocity at step 8
    assert np.abs(u_prev.cpu().numpy() - u8).max() < 1e-12
    # a second call without stepping measures no change
    assert sim.velocity_change(u_prev).item() == 0.0
    for comp, n in ((0, a8), (1, b8)):
        bg = float(n.min())
        com = sim.centre_of_mass(comp, bg).cpu().numpy()
        w = (n - bg).reshape(shape[::-1])
        z, y, x = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]), indexing="ij")
        W = w.sum()
        np.testing.assert_allclose(com[:3], [(w * x).sum() / W, (w * y).sum() / W, (w * z).sum() / W], rtol=1e-12)
        assert com[3] == pytest.approx(W, rel=1e-12)


@pytest.mark.parametrize("storage", ["F32", "F16"])
def test_retired_member_keeps_its_state(B, storage):
    st = getattr(B, f"SC_STORE_{storage}")
    sides, sets = (32, 40, 36), []
    for k, L in enumerate(sides):
        kw = dict(G=2.5, G_self=(0.0, 0.0) if k % 2 == 0 else (-0.4, 0.0), tau=(1.0, 1.0))
        f = S.droplet((L, L, L), (L // 2,) * 3, L / 4.0, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=300 + k)
        sets.append((B.make_params((L, L, L), psi_self=1, storage=st, tile_z=16, **kw), f, kw, L))
    batch = B.Batch([x[0] for x in sets], [x[1] for x in sets])
    batch.step(10)
    batch.retire(1)
    assert batch.active == 2
    batch.step(45)  # crosses a graph replay (32 steps) on the rebuilt work list
    batch.retire(1)  # retiring twice changes nothing
    steps = {0: 55, 1: 10, 2: 55}
    for k, (p, f, kw, L) in enumerate(sets):
        lone = B.Simulation(B.make_params((L, L, L), psi_self=1, storage=st, tile_z=16, variant=1, **kw), *f)
        lone.step(steps[k])
        np.testing.assert_array_equal(batch.members[k].state().cpu().numpy(), lone.state().cpu().numpy())
        assert batch.members[k].launches == steps[k]
    batch.retire(0)
    batch.retire(2)
    assert batch.active == 0
    before = batch.members[2].state().cpu().numpy()
    batch.step(7)  # nothing left to step
    np.testing.assert_array_equal(batch.members[2].state().cpu().numpy(), before)
