"""The batched radius sweep: lattices of uneven sizes and parameters stepped
together, one launch per time step (replayed from a CUDA graph) or, for the
staged kernel, one persistent launch per 32 steps.  Each
member must match the same lattice stepped on its own, bit for bit (same
kernel body and arithmetic), and the FP64 member must match the oracle."""
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


def droplet_set(B, storage):
    """Four odd-sized cubes (side 2 floor(2R) + 1), alternately symmetric and asymmetric."""
    out = []
    for k, R in enumerate((4.0, 5.5, 7.0, 8.5)):
        L = 2 * int(2 * R) + 1
        shape = (L, L, L)
        sym = k % 2 == 0
        kw = dict(G=2.5, G_self=(0.0, 0.0) if sym else (-0.4, 0.0), tau=(1.0, 1.0))
        p = B.make_params(shape, lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=storage, tile_z=7, **kw)
        f = S.droplet(shape[::-1], (L // 2,) * 3, R, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=100 + k)
        out.append((p, f, kw, shape))
    return out


@pytest.mark.parametrize("nsteps", [9, 70])
def test_batch_members_equal_single_runs(B, nsteps):
    sets = droplet_set(B, B.SC_STORE_F32)
    batch = B.Batch([s[0] for s in sets], [s[1] for s in sets])
    batch.step(nsteps)
    assert batch.launches == nsteps
    for (p, f, kw, shape), m in zip(sets, batch.members):
        single = B.Simulation(B.make_params(shape, lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP,
                                            storage=B.SC_STORE_F32, tile_z=7, variant=1, **kw), *f)
        single.step(nsteps)
        np.testing.assert_array_equal(m.populations().cpu().numpy(), single.populations().cpu().numpy())


@pytest.mark.parametrize("storage", ["F32", "F16"])
def test_staged_batch_members_equal_single_runs(B, storage):
    """Sides 4 ceil(R) (multiples of 4, partial x tiles): every member can take
    the staged kernel, so the batch steps with the batched staged kernel; its
    members equal lone runs of the generic kernel bit for bit."""
    st = getattr(B, f"SC_STORE_{storage}")
    sets = []
    for k, R in enumerate((8.0, 9.5, 11.0, 16.0)):
        L = 4 * int(np.ceil(R))
        kw = dict(G=2.5, G_self=(0.0, 0.0) if k % 2 == 0 else (-0.4, 0.0), tau=(1.0, 1.0))
        p = B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=st, tile_z=16, **kw)
        f = S.droplet((L, L, L), (L // 2,) * 3, R, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=200 + k)
        sets.append((p, f, kw, L))
    batch = B.Batch([s_[0] for s_ in sets], [s_[1] for s_ in sets])
    assert batch.staged and batch.persistent
    batch.step(37)
    for (p, f, kw, L), m in zip(sets, batch.members):
        single = B.Simulation(B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=st,
                                            tile_z=16, variant=1, **kw), *f)
        single.step(37)
        np.testing.assert_array_equal(m.state().cpu().numpy(), single.state().cpu().numpy())


def test_batch_fp64_member_matches_oracle(B):
    sets = droplet_set(B, B.SC_STORE_F64)
    batch = B.Batch([s[0] for s in sets], [s[1] for s in sets])
    batch.step(12)
    p, f, kw, shape = sets[1]
    op = oracle.Params(shape=shape, lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, **kw)
    ref = oracle.step(op, oracle.init(op, *f), 12)
    got = batch.members[1].populations().cpu().numpy()
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_batch_member_analysis_and_guard(B):
    sets = droplet_set(B, B.SC_STORE_F32)
    batch = B.Batch([s[0] for s in sets], [s[1] for s in sets])
    batch.step(33)
    m = batch.members[3]
    L = m.shape[0]
    rows, out = B.surface_of_tension(m, (L // 2,) * 3, 0.5)
    assert np.isfinite(out.cpu().numpy()[:4]).all()
    with pytest.raises(B.ScError) as e:
        m.step(1)
    assert e.value.status == B.SC_EINVAL


def test_staged_batch_fp64_member_matches_oracle(B):
    """FP64 storage, sides 4 ceil(R) (the staged kernel, partial x tiles): a batch member
    against the FP64 oracle, one step and twelve."""
    sets = []
    for k, R in enumerate((8.0, 9.0)):
        L = 4 * int(np.ceil(R))
        kw = dict(G=2.5, G_self=(0.0, 0.0) if k == 0 else (-0.4, 0.1), tau=(1.0, 0.9))
        f = S.droplet((L, L, L), (L // 2,) * 3, R, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=400 + k)
        sets.append((B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F64,
                                   tile_z=8, **kw), f, kw, L))
    batch = B.Batch([x[0] for x in sets], [x[1] for x in sets])
    assert batch.staged
    batch.step(12)
    for (p, f, kw, L), m in zip(sets, batch.members):
        op = oracle.Params(shape=(L, L, L), lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, **kw)
        ref = oracle.step(op, oracle.init(op, *f), 12)
        got = m.populations().cpu().numpy()
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("storage", ["F32", "BF16"])
def test_persistent_batch_equals_per_step_launches(B, storage):
    """More work items than co-resident blocks (tile_z 2: 800 items), so each block
    of the persistent launch takes several items per step.  The batch run as
    persistent launches (tile 32 x 8, one stage, two blocks per SM) equals the same batch run one launch
    per step bit for bit
    (single steps, then whole 32-step runs from an even step, then single steps),
    and member 0 equals a lone run; member 1 has tau != 1 (the general collision)."""
    st = getattr(B, f"SC_STORE_{storage}")
    sets = []
    for k, L in enumerate((64, 48)):
        kw = dict(G=2.5, G_self=(0.0, 0.0) if k == 0 else (-0.4, 0.0), tau=(1.0, 1.0) if k == 0 else (0.9, 1.0))
        f = S.droplet((L, L, L), (L // 2,) * 3, L / 4, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=500 + k)
        sets.append((B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=st, tile_y=8,
                                   tile_z=2, stages=1, blocks_per_sm=2, **kw), f, kw, L))
    states = []
    for persistent in (True, False):
        batch = B.Batch([x[0] for x in sets], [x[1] for x in sets])
        assert batch.staged
        batch.persistent = persistent
        assert batch.persistent == persistent
        batch.step(3)
        batch.step(66)
        assert batch.launches == 69
        for m in batch.members:
            m.sync()  # a status word with a timed-out barrier raises here
        states.append([m.state().cpu().numpy() for m in batch.members])
    for a, b in zip(*states):
        np.testing.assert_array_equal(a, b)
    p, f, kw, L = sets[0]
    lone = B.Simulation(B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=st, tile_z=16,
                                      variant=1, **kw), *f)
    lone.step(69)
    np.testing.assert_array_equal(states[0][0], lone.state().cpu().numpy())


def test_bounded_wait_runs_out_and_reports_timeout(B):
    """The persistent launch's grid-barrier wait is bounded: a wait for an arrival that never comes
    (the library's self-test, one block) runs out after its polls, sc_sync reports SC_ETIMEOUT once,
    and the context's state and stepping are untouched (bit-equal to a context that never waited)."""
    L = 32
    kw = dict(G=2.5, G_self=(0.0, 0.0), tau=(1.0, 1.0))
    f = S.droplet((L, L, L), (L // 2,) * 3, 8.0, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=700)
    p = B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F32, **kw)
    sim, ref = B.Simulation(p, *f), B.Simulation(p, *f)
    sim.step(3)
    B.sc_selftest_wait_timeout(sim.ctx, 4096)
    with pytest.raises(B.ScError) as e:
        sim.sync()
    assert e.value.status == B.SC_ETIMEOUT
    sim.sync()  # the flag was cleared
    sim.step(5)
    ref.step(8)
    sim.sync()
    ref.sync()
    np.testing.assert_array_equal(sim.state().cpu().numpy(), ref.state().cpu().numpy())


def test_tune_batch_times_both_launch_forms(B):
    """The batch autotuner times every candidate block shape in both launch forms of a staged batch
    (persistent, and one launch per step), returns (tile_y, tile_z, stages, blocks_per_sm, persistent),
    and a batch with the tuned shape and form equals the default batch bit for bit."""
    from paper_2112_02574_gb300 import tune

    sets = []
    for k, L in enumerate((32, 40)):
        kw = dict(G=2.5, G_self=(0.0, 0.0) if k == 0 else (-0.4, 0.0), tau=(1.0, 1.0))
        f = S.droplet((L, L, L), (L // 2,) * 3, L / 4, n_in=0.85, n_out=0.15, amplitude=1e-3, seed=800 + k)
        sets.append((B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F32,
                                   **kw), f))
    plist, fields = [x[0] for x in sets], [x[1] for x in sets]
    cands = [(8, 0, 1, 3), (4, 0, 1, 3)]
    best, ms, table = tune.tune_batch(plist, fields, cands, steps=32)
    assert len(best) == 5 and best[:4] in cands and ms > 0
    assert sorted(c for c, _ in table) == sorted(c + (p,) for c in cands for p in (True, False))
    tuned = B.Batch([tune.with_config(p, best) for p in plist], fields)
    tuned.persistent = best[4]
    default = B.Batch(plist, fields)
    tuned.step(40)
    default.step(40)
    for a, b in zip(tuned.members, default.members):
        np.testing.assert_array_equal(a.state().cpu().numpy(), b.state().cpu().numpy())
