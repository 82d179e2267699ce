"""GPU parity: the fused CUDA step and the analysis kernels, called through the
C ABI, against the FP64 CPU oracle on the same seeded inputs.

Tolerances
* FP64 storage + FP64 collision: the same arithmetic as the oracle in another
  order -> max |f_gpu - f_orc| <= 1e-13 max |f| after the steps run here.
* FP32 storage (deviations from the rest equilibrium) + FP32 collision:
  densities and populations within 1e-6 relative of the FP64 oracle (max-norm,
  normalised by the field's max); the velocity within 1e-5 relative to max |u|
  (FP32_U_REL below: u is a small difference of O(0.1) populations, each
  stored with an FP32 rounding, so its error is set by that absolute scale).
* Integer-like results (counts, bitwise symmetries, tile independence in FP64,
  checkpoint/resume) are exact."""
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


def setup(B, shape, storage, lattice=1, stencil=0, psi=1, tau=(1.0, 0.9), G=2.5, G_self=(-0.4, 0.0), amp=1e-3,
          radius=None, tile_y=0, tile_z=0, n_in=0.85, n_out=0.15, seed=S.DEFAULT_SEED):
    nx, ny, nz = shape
    centre = (nx // 2, ny // 2, nz // 2)
    R = radius if radius is not None else min(nx, ny, nz if nz > 1 else ny) / 4
    nA0, nB0 = S.droplet(shape[::-1], centre, R, n_in=n_in, n_out=n_out, amplitude=amp, seed=seed)
    p = B.make_params(shape, lattice=lattice, stencil=stencil, psi_self=psi, storage=storage, tau=tau, G=G,
                      G_self=G_self, tile_y=tile_y, tile_z=tile_z)
    op = oracle.Params(shape=shape, lattice=lattice, stencil=stencil, psi_self=psi, tau=tau, G=G, G_self=G_self)
    return B.Simulation(p, nA0, nB0), op, nA0, nB0


# FP32 storage: the common velocity of Eq. u relative to max|u|.  u is a difference of populations of
# order w_i n ~ 0.03-0.3, each stored in FP32 as a deviation of up to M ~ 0.45 w_1 (the interface) and
# rounded once per step (relative 2^-24), with a few more FP32 roundings of the same size in the
# collision; after k steps the ~20 populations entering u carry independent errors of about
# sqrt(k) 4 ulp(M) ~ 3.5 x 4 x 1.5e-9 = 2e-8 each, so |du| ~ sqrt(20) x 2e-8 ~ 1e-7 in lattice units,
# i.e. 1e-5 relative to max|u| ~ 1e-2 (measured over the cases here: 0.8e-6 .. 4.5e-6).  The 1e-6 of
# the densities and populations cannot hold for u, a small difference of large terms.
FP32_U_REL = 1e-5


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


CASES = [
    # (shape, lattice, stencil, psi, G_self) -- every shape spans >1 tile in x and y with a ragged tail;
    # by default the D3Q19 / E4 shapes take the staged kernel where nx >= 32 is a multiple of the
    # storage's chunk sites (FP64: any nx, so also the partial x tiles of nx = 37 and 70), the others
    # the generic one
    ((64, 21, 19), 1, 0, 1, (-0.4, 0.0)),
    ((96, 10, 7), 1, 0, 0, (0.0, 0.0)),
    ((37, 11, 19), 1, 0, 1, (-0.4, 0.0)),
    ((70, 9, 6), 1, 0, 0, (0.0, 0.0)),
    ((35, 10, 18), 1, 1, 1, (-0.4, 0.2)),
    ((70, 45, 1), 0, 0, 0, (0.0, 0.0)),
    ((33, 13, 1), 0, 0, 1, (-0.3, 0.0)),
    # whole 32-site x tiles and whole y tiles of every tile_y (the bench workload's tiling)
    ((64, 16, 12), 1, 0, 1, (-0.4, 0.0)),
]


@pytest.mark.parametrize("shape,lattice,stencil,psi,G_self", CASES)
def test_fp64_step_matches_oracle(B, shape, lattice, stencil, psi, G_self):
    sim, op, nA0, nB0 = setup(B, shape, B.SC_STORE_F64, lattice, stencil, psi, G_self=G_self)
    sim.step(12)
    sim.sync()
    f = sim.populations().cpu().numpy()
    ref = oracle.step(op, oracle.init(op, nA0, nB0), 12)
    assert rel(f, ref) < 1e-13
    nA, nB, u = sim.moments()
    oA, oB, ou = oracle.moments(op, ref)
    assert rel(nA.cpu(), oA) < 1e-13 and rel(nB.cpu(), oB) < 1e-13
    assert np.abs(u.cpu().numpy() - ou).max() < 1e-13 * max(1.0, np.abs(ou).max())


@pytest.mark.parametrize("shape,lattice,stencil,psi,G_self", CASES)
def test_fp32_step_matches_oracle(B, shape, lattice, stencil, psi, G_self):
    sim, op, nA0, nB0 = setup(B, shape, B.SC_STORE_F32, lattice, stencil, psi, G_self=G_self)
    sim.step(12)
    sim.sync()
    ref = oracle.step(op, oracle.init(op, nA0, nB0), 12)
    nA, nB, u = sim.moments()
    oA, oB, ou = oracle.moments(op, ref)
    assert rel(nA.cpu(), oA) < 1e-6 and rel(nB.cpu(), oB) < 1e-6
    eu = rel(u.cpu().numpy(), ou)  # max |u_gpu - u_orc| / max |u_orc|
    print(f"FP32 storage, 12 steps: u within {eu:.2e} of max|u| = {np.abs(ou).max():.2e}")
    assert eu < FP32_U_REL
    assert rel(sim.populations().cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("shape,lattice,stencil,psi,G_self", CASES)
@pytest.mark.parametrize("storage", ["F64", "F32"])
def test_tau_one_step_matches_oracle(B, shape, lattice, stencil, psi, G_self, storage):
    """tau_A = tau_B = 1: the kernels' instantiation that carries a site's momentum sums instead of its
    populations from its density sum to its collision (generic, staged, E4, E6, D2Q9) against the
    oracle, at the tolerances of the general form (FP64 1e-13, FP32 1e-6 and FP32_U_REL)."""
    st = getattr(B, f"SC_STORE_{storage}")
    sim, op, nA0, nB0 = setup(B, shape, st, lattice, stencil, psi, tau=(1.0, 1.0), G_self=G_self)
    sim.step(12)
    sim.sync()
    ref = oracle.step(op, oracle.init(op, nA0, nB0), 12)
    nA, nB, u = sim.moments()
    oA, oB, ou = oracle.moments(op, ref)
    tol = 1e-13 if storage == "F64" else 1e-6
    assert rel(sim.populations().cpu().numpy(), ref) < tol
    assert rel(nA.cpu(), oA) < tol and rel(nB.cpu(), oB) < tol
    assert rel(u.cpu().numpy(), ou) < (1e-12 if storage == "F64" else FP32_U_REL)


def test_config1_d2q9_2000_steps(B):
    """The 64x64 D2Q9 droplet workload (G c_s^2 = 1.4, psi = n, tau = 1), 2000
    steps, FP64 and FP32 storage against the FP64 oracle.  The minority density
    dips slightly below zero around step 200 in the oracle too (psi = n keeps
    the method defined there); it recovers by step 2000."""
    shape = (64, 64, 1)
    nA0, nB0 = S.droplet((1, 64, 64), (32, 32, 0), 12.0)
    kw = dict(tau=(1.0, 1.0), G=4.2, G_self=(0.0, 0.0))
    op = oracle.Params(shape=shape, lattice=0, psi_self=0, **kw)
    ref = oracle.step(op, oracle.init(op, nA0, nB0), 2000)
    oA, oB, ou = oracle.moments(op, ref)
    # FP32: each step adds a relative round-off of about eps_32 = 6e-8 to the stored
    # populations, and over T steps it accumulates at most ~T eps_32: 2000 x 6e-8 = 1.2e-4
    for storage, tol in ((B.SC_STORE_F64, 1e-12), (B.SC_STORE_F32, 2000 * 6e-8)):
        p = B.make_params(shape, lattice=0, psi_self=0, storage=storage, **kw)
        sim = B.Simulation(p, nA0, nB0)
        sim.step(2000)
        sim.sync()
        nA, nB, u = sim.moments()
        assert rel(nA.cpu(), oA) < tol, storage
        assert rel(nB.cpu(), oB) < tol, storage
        assert np.abs(u.cpu().numpy() - ou).max() < tol  # lattice units (relative to the lattice speed)


@pytest.mark.parametrize("storage", ["F64", "F32"])
def test_tiling_does_not_change_results(B, storage):
    """Block shape (tile rows, planes per block) only reorders work: results are bitwise equal."""
    st = getattr(B, f"SC_STORE_{storage}")
    outs = []
    for ty, tz in ((4, 16), (1, 1), (2, 5), (8, 3)):
        sim, *_ = setup(B, (45, 19, 23), st, tile_y=ty, tile_z=tz)
        sim.step(7)
        sim.sync()
        outs.append(sim.state().cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("storage", ["F32", "F16", "BF16", "F64"])
def test_staged_kernel_equals_generic_bitwise(B, storage):
    """The cp.async-staged kernel moves data differently but sums and collides in
    the same order as the generic kernel: the states agree bit for bit for every
    tile shape, pipeline depth and register budget."""
    st = getattr(B, f"SC_STORE_{storage}")
    outs = []
    # tile_z 0: the balanced z split (columns cut into K or K + 1 chunks, 1-D grid)
    configs = [(1, 4, 5, 0, 0), (2, 4, 3, 2, 2), (2, 4, 3, 1, 3), (2, 4, 7, 2, 3), (2, 4, 1, 1, 2), (2, 4, 0, 2, 2)]
    if storage != "F64":
        configs += [(2, 8, 7, 2, 1), (2, 8, 2, 1, 2), (2, 8, 13, 2, 2), (2, 8, 5, 1, 1), (2, 8, 0, 1, 2),
                    (2, 16, 7, 1, 1), (2, 16, 0, 1, 1)]
    if storage in ("F16", "BF16"):
        configs += [(2, 16, 4, 2, 1)]
    for variant, ty, tz, ns, mb in configs:
        sim2 = B.Simulation(B.make_params((96, 19, 13), psi_self=1, storage=st, tau=(1.0, 0.9), G=2.5,
                                          G_self=(-0.4, 0.1), tile_y=ty, tile_z=tz, variant=variant, stages=ns,
                                          blocks_per_sm=mb),
                            *S.droplet((13, 19, 96), (48, 9, 6), 3.25, n_in=0.85, n_out=0.15, amplitude=1e-3))
        sim2.step(9)
        sim2.sync()
        outs.append(sim2.state().cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("storage", ["F32", "F16"])
@pytest.mark.parametrize("G_self", [(-0.4, 0.0), (0.0, 0.0)])
def test_balanced_z_split_equals_generic(B, storage, G_self):
    """A box whose balanced split gives columns of unequal chunk counts (on a
    152-SM GPU: FP32, three blocks per SM, 456 blocks over 30 columns, K = 15
    with 6 columns of 16 chunks; FP16 304 blocks over 15 columns, K = 20 with 4
    columns of 21):
    same state as the generic kernel, bit for bit; with and without a self
    coupling (without one the staged launch leaves the psi ring out)."""
    st = getattr(B, f"SC_STORE_{storage}")
    shape = (96, 40, 128)
    f = S.droplet(shape[::-1], (48, 20, 64), 12.0, n_in=0.85, n_out=0.15, amplitude=1e-3)
    outs = []
    for variant, tz in ((1, 32), (2, 0)):
        sim = B.Simulation(B.make_params(shape, psi_self=1, storage=st, G=2.5, G_self=G_self, tile_z=tz,
                                         variant=variant), *f)
        sim.step(5)
        sim.sync()
        if variant == 2:
            cfg = sim.step_config
            import torch

            sms = torch.cuda.get_device_properties(0).multi_processor_count
            assert cfg["variant"] == 2 and cfg["zsplit_k"] > 0 and cfg["blocks"] % sms == 0
        outs.append(sim.state().cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])


@pytest.mark.parametrize("storage", ["F32", "F16", "F64"])
@pytest.mark.parametrize("stencil", [0, 1])
def test_generic_balanced_z_split_equals_fixed_chunks(B, storage, stencil):
    """The generic kernel's balanced z split (1-D grid, columns cut into K or K + 1
    chunks of unequal length) against fixed 5-plane chunks on a 3-D grid: the same
    state bit for bit, E4 and E6 (a z reach of one and two planes)."""
    import torch

    st = getattr(B, f"SC_STORE_{storage}")
    shape = (96, 40, 128)
    f = S.droplet(shape[::-1], (48, 20, 64), 12.0, n_in=0.85, n_out=0.15, amplitude=1e-3)
    outs = []
    for tz in (5, 0):
        sim = B.Simulation(B.make_params(shape, stencil=stencil, psi_self=1, storage=st, G=2.5, G_self=(-0.4, 0.1),
                                         tile_z=tz, variant=1), *f)
        sim.step(5)
        sim.sync()
        cfg = sim.step_config
        assert cfg["variant"] == 1
        if tz == 0:
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            assert cfg["zsplit_k"] > 0 and cfg["blocks"] % sms == 0, cfg
        outs.append(sim.state().cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])


@pytest.mark.parametrize("storage", ["F32", "F16", "BF16", "F64"])
@pytest.mark.parametrize("nx", [32, 36, 44, 100])
def test_staged_partial_x_tiles_equal_generic(B, storage, nx):
    """Partial last x tile (nx not a multiple of 32) and a single tile narrower
    than the copy window: the staged kernel's per-chunk periodic wrap gives the
    generic kernel's state bit for bit."""
    st = getattr(B, f"SC_STORE_{storage}")
    shape = (nx, 11, 6)
    outs = []
    for variant in (1, 2):
        sim = B.Simulation(B.make_params(shape, psi_self=1, storage=st, G=2.5, G_self=(-0.4, 0.1), tau=(1.0, 0.8),
                                         tile_z=4, variant=variant),
                           *S.droplet(shape[::-1], (nx // 2, 5, 3), 3.0, n_in=0.85, n_out=0.15, amplitude=1e-3))
        sim.step(6)
        sim.sync()
        outs.append(sim.state().cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])


@pytest.mark.parametrize("storage", ["F32", "F16"])
@pytest.mark.parametrize("nz", [1, 2, 3])
def test_staged_thin_z_equals_generic(B, storage, nz):
    """Periodic wrap of the staged kernel's plane windows when the box is thinner
    than the z reach of a block (nz < 3): same state as the generic kernel."""
    st = getattr(B, f"SC_STORE_{storage}")
    shape = (64, 9, nz)
    outs = []
    for variant in (1, 2):
        sim = B.Simulation(B.make_params(shape, psi_self=1, storage=st, G=2.5, G_self=(-0.4, 0.0), tile_y=4,
                                         tile_z=2, variant=variant),
                           *S.droplet(shape[::-1], (32, 4, 0), 3.0, n_in=0.85, n_out=0.15, amplitude=1e-3))
        sim.step(7)
        sim.sync()
        outs.append(sim.state().cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])


@pytest.mark.parametrize("storage,u", [("F16", 2.0**-11), ("BF16", 2.0**-8)])
@pytest.mark.parametrize("staged", [False, True])
def test_sixteen_bit_storage_against_oracle(B, storage, u, staged):
    """16-bit deviation storage against the FP64 oracle after k steps.  Each step
    rounds every stored deviation from the site's rest equilibrium once, to
    within u |g| (u the unit roundoff: 2^-11 FP16, 2^-8 BF16; FP16 carries a
    power-of-two scale, so no value leaves the normal range), and the FP32
    collision adds errors far below that.  Independent roundings of the 19
    populations that feed each collision add like a random walk, so after k
    steps the populations stay within 2 k u M of the oracle, M the largest
    deviation |f_i - w_i n| of the oracle's state; the densities likewise.
    The run prints the measured fraction of that bound."""
    shape = (64, 12, 10)
    k = 10
    nA0, nB0 = S.droplet(shape[::-1], (32, 6, 5), 3.0, n_in=0.85, n_out=0.15, amplitude=1e-3)
    kw = dict(tau=(1.0, 0.9), G=2.5, G_self=(-0.4, 0.0))
    p = B.make_params(shape, psi_self=1, storage=getattr(B, f"SC_STORE_{storage}"), variant=2 if staged else 1, **kw)
    sim = B.Simulation(p, nA0, nB0)
    sim.step(k)
    sim.sync()
    assert sim.step_config["variant"] == (2 if staged else 1)
    op = oracle.Params(shape=shape, lattice=1, psi_self=1, **kw)
    f_orc = oracle.step(op, oracle.init(op, nA0, nB0), k)
    _, w = oracle.velocity_set(1)
    n_orc = f_orc.sum(axis=1)  # [2, N]
    M = float(np.abs(f_orc - w[None, :, None] * n_orc[:, None, :]).max())
    f_gpu = sim.populations().cpu().numpy()
    err_f = float(np.abs(f_gpu - f_orc).max())
    nA, nB, _ = sim.moments(with_u=False)
    err_n = max(float(np.abs(nA.cpu().numpy() - n_orc[0]).max()), float(np.abs(nB.cpu().numpy() - n_orc[1]).max()))
    bound = 2 * k * u * M
    print(f"{storage} staged={staged}: max |df| = {err_f:.3e} ({err_f / bound:.3f} of 2 k u M), "
          f"max |dn| = {err_n:.3e} ({err_n / bound:.3f}), M = {M:.3e}")
    assert err_f <= bound
    assert err_n <= bound


@pytest.mark.parametrize("storage", ["F32", "F16"])
def test_tuner_choice_changes_speed_only(B, storage):
    """The single-lattice autotuner times every candidate it lists (the library
    default first) and returns the fastest; that configuration computes the
    default's state bit for bit."""
    from paper_2112_02574_gb300 import tune

    st = getattr(B, f"SC_STORE_{storage}")
    shape = (64, 24, 40)
    f = S.droplet(shape[::-1], (32, 12, 20), 6.0, n_in=0.85, n_out=0.15, amplitude=1e-3)
    kw = dict(psi_self=1, storage=st, tau=(1.0, 0.9), G=2.5, G_self=(-0.4, 0.0))
    p = B.make_params(shape, **kw)
    best, ms, table = tune.tune_step(p, *f, steps=8, warmup=2)
    assert [c for c, _ in table] == tune.candidates_for(p)
    assert all(t > 0 for _, t in table) and ms == min(t for _, t in table)
    outs = []
    for variant, ty, tz, ns, mb in ((0, 0, 0, 0, 0), best):
        sim = B.Simulation(B.make_params(shape, tile_y=ty, tile_z=tz, variant=variant, stages=ns, blocks_per_sm=mb,
                                         **kw), *f)
        sim.step(7)
        sim.sync()
        outs.append(sim.state().cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])


def test_swap_symmetry_bitwise(B):
    """Section 2: G_AA = G_BB and tau_A = tau_B make A <-> B an exact symmetry."""
    shape = (40, 12, 9)
    nA0, nB0 = S.droplet(shape[::-1], (20, 6, 4), 3.0, n_in=0.85, n_out=0.15)
    kw = dict(lattice=1, psi_self=1, storage=B.SC_STORE_F32, tau=(0.9, 0.9), G=2.5, G_self=(-0.3, -0.3))
    a = B.Simulation(B.make_params(shape, **kw), nA0, nB0)
    b = B.Simulation(B.make_params(shape, **kw), nB0, nA0)
    a.step(25)
    b.step(25)
    fa, fb = a.populations().cpu().numpy(), b.populations().cpu().numpy()
    np.testing.assert_array_equal(fa[0], fb[1])
    np.testing.assert_array_equal(fa[1], fb[0])


def test_uniform_mixture_stays_uniform(B):
    shape = (40, 7, 6)
    for storage in (B.SC_STORE_F32, B.SC_STORE_F16, B.SC_STORE_BF16):
        p = B.make_params(shape, psi_self=1, storage=storage, tau=(0.7, 1.3), G=3.0, G_self=(-0.5, 0.2))
        sim = B.Simulation(p, *S.uniform(shape[::-1], 0.37, 0.71))
        sim.step(30)
        f = sim.populations().cpu().numpy()
        assert not np.ptp(f, axis=2).any()
        nA, nB, u = sim.moments()
        assert not u.cpu().numpy().any()


def test_conservation(B):
    """Section 2: per-component mass exactly conserved (FP32 storage: drift at
    round-off level); total momentum conserved for tau_A = tau_B."""
    sim, op, nA0, nB0 = setup(B, (48, 20, 16), B.SC_STORE_F32, tau=(0.9, 0.9), amp=1e-2)
    t0 = sim.totals().cpu().numpy()
    sim.step(200)
    t1 = sim.totals().cpu().numpy()
    assert abs(t0[0] - nA0.sum()) < 1e-7 * nA0.sum()
    assert np.abs(t1[:2] - t0[:2]).max() < 1e-6 * t0[:2].max()
    assert np.abs(t1[2:]).max() < 1e-6 * t0[:2].sum()


def test_checkpoint_resume_bitwise(B):
    sim, *_ = setup(B, (40, 12, 10), B.SC_STORE_F32)
    sim.step(5)
    snap = sim.state().clone()
    sim.step(9)
    a = sim.state().cpu().numpy()
    sim.set_state(snap)
    sim.step(9)
    np.testing.assert_array_equal(sim.state().cpu().numpy(), a)


def test_set_get_populations_roundtrip(B):
    sim, op, nA0, nB0 = setup(B, (35, 9, 7), B.SC_STORE_F64)
    f = oracle.step(op, oracle.init(op, nA0, nB0), 3)
    sim.set_populations(f)
    g = sim.populations().cpu().numpy()
    assert rel(g, f) < 1e-15
    sim.step(2)
    assert rel(sim.populations().cpu().numpy(), oracle.step(op, f, 2)) < 1e-13


def test_nonpositive_density_is_reported(B):
    """A state with a negative density makes the step set the status word;
    sc_sync returns SC_ENAN (a host-side error code, no device fault)."""
    sim, op, nA0, nB0 = setup(B, (34, 6, 5), B.SC_STORE_F32)
    f = oracle.init(op, nA0, nB0)
    f[0, :, 7] = -0.1
    sim.set_populations(f)
    sim.step(1)
    with pytest.raises(B.ScError) as e:
        sim.sync()
    assert e.value.status == B.SC_ENAN
    sim.sync()  # flag cleared


# ------------------------------------------------------------ analysis path
@pytest.mark.parametrize("lattice,stencil", [(1, 0), (1, 1), (0, 0)])
def test_profiles_match_oracle(B, lattice, stencil):
    shape = (40, 36, 34) if lattice == 1 else (64, 60, 1)
    sim, op, nA0, nB0 = setup(B, shape, B.SC_STORE_F64, lattice, stencil, 1, G_self=(-0.4, 0.1), amp=1e-2)
    sim.step(6)
    f = sim.populations().cpu().numpy()
    oA, oB, _ = oracle.moments(op, f, with_u=False)
    centre = (20.0, 18.0, 17.0) if lattice == 1 else (32.0, 30.0, 0.0)
    for kind, nbins, bw in ((B.SC_PROFILE_RADIAL, 40, 0.5), (B.SC_PROFILE_PLANAR_Z, shape[2], 1.0),
                            (B.SC_PROFILE_AXIS_X, 20, 1.0)):
        got = sim.profile(kind, centre, bw, nbins).cpu().numpy()
        want = oracle.profile(op, oA, oB, kind, centre, bw, nbins)
        np.testing.assert_array_equal(got[:, 5], want[:, 5])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
    for node in ((0, 0, 0), (shape[0] - 1, shape[1] - 1, shape[2] - 1), (3, 5, 0)):
        s = node[0] + shape[0] * (node[1] + shape[1] * node[2])
        assert sim.bulk_pressure(node).item() == pytest.approx(oracle.bulk_pressure(op, oA[s], oB[s]), rel=1e-13)


def test_sigma_minimum_matches_oracle(B):
    import torch

    import oracle.sigma as SG

    r = np.linspace(0.0, 20.0, 81)
    pt = 0.33 - 0.01 * np.exp(-0.5 * (r - 8.0) ** 2) + 0.004 * (r < 8.0)
    rows = np.zeros((90, 6))
    rows[:81, 0] = r
    rows[:81, 2] = pt
    rows[:81, 5] = 1.0
    rows[40, 5] = 0.0  # an empty bin is skipped
    keep = rows[:, 5] > 0
    pio = torch.tensor([0.334, 0.330], dtype=torch.float64, device="cuda")
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    for dim in (3, 2):
        B.sc_sigma_minimum(torch.tensor(rows, device="cuda"), pio, dim, 1.0, 19.0, 0.01, out)
        o = out.cpu().numpy()
        want = SG.surface_of_tension(rows[keep, 0], rows[keep, 2], 0.334, 0.330, dim=dim)
        assert o[0] == pytest.approx(want["dP"], rel=1e-15)
        assert o[1] == pytest.approx(want["C"], rel=1e-13)
        assert o[2] == pytest.approx(want["Rs"], rel=1e-13)
        assert o[3] == pytest.approx(want["sigma_s"], rel=1e-13)
        Rg, sg = SG.argmin_on_grid(rows[keep, 0], rows[keep, 2], 0.334, 0.330, 1.0, 19.0, 0.01, dim=dim)
        assert o[4] == pytest.approx(Rg, rel=1e-9)
        assert o[5] == pytest.approx(sg, rel=1e-9)


def test_sigma0_flat_matches_oracle(B):
    """Section 4: sigma_0 of a slab, the device reduction of the device planar
    profile against the oracle's sum over the oracle's profile (FP64 storage)."""
    import oracle.sigma as SG

    shape = (16, 12, 64)
    nA0, nB0 = S.slab(shape[::-1], 32.0, amplitude=1e-3)
    p = B.make_params(shape, psi_self=1, storage=B.SC_STORE_F64, G=3.6, G_self=(-0.6, 0.0))
    sim = B.Simulation(p, nA0, nB0)
    sim.step(40)
    rows, s0 = B.sigma0_flat(sim)
    op = oracle.Params(shape=shape, lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, G=3.6, G_self=(-0.6, 0.0))
    f = oracle.step(op, oracle.init(op, nA0, nB0), 40)
    oA, oB, _ = oracle.moments(op, f, with_u=False)
    want_rows = oracle.profile(op, oA, oB, oracle.PLANAR_Z, (0.0, 0.0, 0.0), 1.0, shape[2])
    want = SG.sigma0_flat(want_rows[:, 1], want_rows[:, 2])
    assert abs(want) > 1e-3
    assert s0.item() == pytest.approx(want, rel=1e-11)
    g = rows.cpu().numpy()
    assert s0.item() == pytest.approx(SG.sigma0_flat(g[:, 1], g[:, 2]), rel=1e-13)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("fixed", [False, True])
def test_curvature_fit_matches_oracle(B, order, fixed):
    """Eq. sigma_c fit on the device against the oracle's least squares, on noisy
    synthetic (R_s, sigma_s) of A-rich (+R_s) and B-rich (-R_s) droplets."""
    import torch

    import oracle.sigma as SG

    rng = np.random.default_rng(11)
    Rs = np.concatenate([np.linspace(6.0, 40.0, 9), -np.linspace(7.0, 38.0, 7)])
    s0, delta, rig = 0.0712, 0.41, 1.3
    sig = s0 * (1 - 2 * delta / Rs + rig / Rs**2) * (1 + 1e-4 * rng.standard_normal(Rs.size))
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    sig0 = dev([s0 * 1.001]) if fixed else None
    out = B.curvature_fit(dev(Rs), dev(sig), order=order, sigma0=sig0).cpu().numpy()
    want = SG.curvature_fit(Rs, sig, order=order, sigma0=s0 * 1.001 if fixed else None)
    assert out[0] == pytest.approx(want["sigma0"], rel=1e-10)
    assert out[1] == pytest.approx(want["delta"], rel=1e-8)
    if order == 2:
        assert out[2] == pytest.approx(want["rigidity"], rel=1e-7)
    else:
        assert np.isnan(out[2])
    x = 1.0 / Rs
    model = want["sigma0"] * (1 - 2 * want["delta"] * x + (want.get("rigidity", 0.0)) * x**2)
    assert out[3] == pytest.approx(np.sqrt(np.mean((model - sig) ** 2)), rel=1e-6)


def test_run_host_matches_device_path(B):
    import torch

    shape = (40, 12, 10)
    nA0, nB0 = S.droplet(shape[::-1], (20, 6, 5), 3.0, n_in=0.85, n_out=0.15)
    p = B.make_params(shape, psi_self=1, storage=B.SC_STORE_F32, tau=(1.0, 0.9), G=2.5, G_self=(-0.4, 0.0))
    ws = torch.empty(B.sc_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    hA = torch.from_numpy(nA0.reshape(-1)).pin_memory()
    hB = torch.from_numpy(nB0.reshape(-1)).pin_memory()
    oA = torch.empty_like(hA).pin_memory()
    oB = torch.empty_like(hB).pin_memory()
    B.sc_run_host(p, hA, hB, 11, oA, oB, ws)
    sim = B.Simulation(p, nA0, nB0)
    sim.step(11)
    nA, nB, _ = sim.moments(with_u=False)
    np.testing.assert_array_equal(oA.numpy(), nA.cpu().numpy())
    np.testing.assert_array_equal(oB.numpy(), nB.cpu().numpy())


def test_step_graph_replay_equals_plain_launches(B):
    """Runs of 32 steps replay a captured CUDA graph; stepping 1 + 70 + 3 steps (graph
    replays and plain launches mixed, odd start parity included) gives the state of 74
    plain single steps, bit for bit, and counts every step as a launch."""
    shape = (64, 21, 19)
    f = S.droplet(shape[::-1], (32, 10, 9), 4.0, n_in=0.85, n_out=0.15, amplitude=1e-3)
    p = B.make_params(shape, psi_self=1, storage=B.SC_STORE_F32, G=2.5, G_self=(-0.4, 0.0))
    a, b = B.Simulation(p, *f), B.Simulation(p, *f)
    for n in (1, 70, 3):
        a.step(n)
    for _ in range(74):
        b.step(1)
    np.testing.assert_array_equal(a.state().cpu().numpy(), b.state().cpu().numpy())
    assert a.launches == 74 and b.launches == 74


@pytest.mark.parametrize("kind", ["RADIAL", "AXIS_X"])
def test_surface_of_tension_matches_oracle(B, kind):
    """sc_surface_of_tension in one call (section 3: Eqs. gen_sigma, gen_d_sigma and the minimum;
    section 4: P_in at the centre node, P_out at the far corner) against the oracle's profile, Eq.
    bulkp at those nodes and the oracle's closed-form and grid minima, FP64 storage."""
    import torch

    import oracle.sigma as SG

    shape = (36, 34, 38)
    sim, op, nA0, nB0 = setup(B, shape, B.SC_STORE_F64, 1, 0, 1, G=3.6, G_self=(-0.6, 0.0), amp=1e-2, radius=8.0,
                              n_in=0.95, n_out=0.05)
    sim.step(300)
    f = sim.populations().cpu().numpy()
    oA, oB, _ = oracle.moments(op, f, with_u=False)
    k = getattr(B, f"SC_PROFILE_{kind}")
    nbins = 34 if kind == "RADIAL" else 18  # min(shape) / 2 / 0.5 and nx / 2
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    rows = torch.empty((nbins, 6), dtype=torch.float64, device="cuda")
    B.sc_surface_of_tension(sim.ctx, k, None, 0.5, 0, 0.0, 0.0, 0.0, out, rows)  # all defaults
    o = out.cpu().numpy()
    centre = (18.0, 17.0, 19.0)
    want_rows = oracle.profile(op, oA, oB, k, centre, 0.5 if kind == "RADIAL" else 1.0, nbins)
    np.testing.assert_array_equal(rows.cpu().numpy()[:, 5], want_rows[:, 5])
    np.testing.assert_allclose(rows.cpu().numpy(), want_rows, rtol=1e-12, atol=1e-14)
    c = 18 + 36 * (17 + 34 * 19)
    p_in, p_out = oracle.bulk_pressure(op, oA[c], oB[c]), oracle.bulk_pressure(op, oA[-1], oB[-1])
    r, _, pt, _, _ = SG.clean_profile(want_rows)
    want = SG.surface_of_tension(r, pt, p_in, p_out)
    assert want["dP"] > 1e-3 and (kind == "AXIS_X" or 4.0 < want["Rs"] < 12.0)  # a formed droplet
    assert o[6] == pytest.approx(p_in, rel=1e-13) and o[7] == pytest.approx(p_out, rel=1e-13)
    for i, key in enumerate(("dP", "C", "Rs", "sigma_s")):
        assert o[i] == pytest.approx(want[key], rel=1e-12), key
    r_max = nbins * (0.5 if kind == "RADIAL" else 1.0)
    Rg, sg = SG.argmin_on_grid(r, pt, p_in, p_out, 0.01, r_max, 0.01)
    assert o[4] == pytest.approx(Rg, rel=1e-9) and o[5] == pytest.approx(sg, rel=1e-9)
    # the binding's one-line wrapper gives the same numbers
    _, o2 = B.surface_of_tension(sim, None, 0.5, kind=k)
    np.testing.assert_array_equal(o2.cpu().numpy(), o)


def test_diagnostics_equals_the_separate_calls(B):
    """sc_diagnostics = sc_totals, sc_velocity_change and sc_centre_of_mass in one call, bit for bit;
    NaN where a part is switched off."""
    import torch

    shape = (40, 24, 20)
    sim, *_ = setup(B, shape, B.SC_STORE_F32, amp=1e-2)
    sim.step(5)
    _, _, u0 = sim.moments()
    u_a, u_b = u0.clone(), u0.clone()
    sim.step(4)
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    B.sc_diagnostics(sim.ctx, u_a, 0, 0.15, out)
    tot = sim.totals()
    du = torch.empty(1, dtype=torch.float64, device="cuda")
    B.sc_velocity_change(sim.ctx, u_b, du)
    com = sim.centre_of_mass(0, 0.15)
    want = torch.cat([tot, du, com]).cpu().numpy()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    np.testing.assert_array_equal(u_a.cpu().numpy(), u_b.cpu().numpy())  # u_prev updated alike
    B.sc_diagnostics(sim.ctx, None, -1, 0.0, out)
    o = out.cpu().numpy()
    np.testing.assert_array_equal(o[:5], tot.cpu().numpy())
    assert np.isnan(o[5:]).all()


def test_run_host_sigma_matches_device_path(B):
    """The host-buffer entry point returns the densities and (dP, C, R_s, sigma_s, ...) of the same
    run on the device path, bit for bit."""
    import torch

    shape = (40, 32, 36)
    nA0, nB0 = S.droplet(shape[::-1], (20, 16, 18), 7.0, n_in=0.9, n_out=0.1)
    p = B.make_params(shape, psi_self=1, storage=B.SC_STORE_F32, G=3.6)
    ws = torch.empty(B.sc_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    hA = torch.from_numpy(nA0.reshape(-1)).pin_memory()
    hB = torch.from_numpy(nB0.reshape(-1)).pin_memory()
    oA, oB = torch.empty_like(hA).pin_memory(), torch.empty_like(hB).pin_memory()
    res = torch.empty(8, dtype=torch.float64).pin_memory()
    B.sc_run_host_sigma(p, hA, hB, 70, (20.0, 16.0, 18.0), 0.5, 32, oA, oB, res, ws)
    sim = B.Simulation(p, nA0, nB0)
    sim.step(70)
    _, out = B.surface_of_tension(sim, (20.0, 16.0, 18.0), 0.5, nbins=32)
    nA, nB, _ = sim.moments(with_u=False)
    np.testing.assert_array_equal(res.numpy(), out.cpu().numpy())
    np.testing.assert_array_equal(oA.numpy(), nA.cpu().numpy())
    np.testing.assert_array_equal(oB.numpy(), nB.cpu().numpy())
    assert res[0] > 0 and np.isfinite(res.numpy()).all()


def test_axis_profile_rejects_more_rows_than_sites(B):
    sim, *_ = setup(B, (20, 12, 10), B.SC_STORE_F64)
    with pytest.raises(B.ScError) as e:
        sim.profile(B.SC_PROFILE_AXIS_X, (10.0, 6.0, 5.0), 1.0, 21)
    assert e.value.status == B.SC_EINVAL
    rows = sim.profile(B.SC_PROFILE_AXIS_X, (10.0, 6.0, 5.0), 1.0, 20).cpu().numpy()
    assert (rows[:, 5] == 1).all()


def test_fp64_step_matches_oracle_over_a_convergence_interval(B):
    """The FP64-storage path, which the reduced-precision errors are measured against, against the
    oracle over one convergence interval of section 4 (2^11 steps) on a 64^3 droplet with asymmetric
    couplings and psi = exp(-1/n).  Both sides are FP64 in a different order of operations; each step
    adds a relative difference of order 2^-52 per value, so after k = 2048 steps the densities are held
    to 1e-12 relative (k x 2.2e-16 = 4.5e-13) and the velocity, a difference of O(0.1) populations
    with max|u| ~ 1e-2, to 1e-11 relative to max|u| (1e-13 in lattice units)."""
    shape = (64, 64, 64)
    sim, op, nA0, nB0 = setup(B, shape, B.SC_STORE_F64, 1, 0, 1, tau=(1.0, 1.0), G=3.6, G_self=(-0.6, 0.0),
                              radius=12.0, n_in=0.95, n_out=0.05)
    sim.step(2048)
    sim.sync()
    nA, nB, u = sim.moments()
    ref = oracle.step(op, oracle.init(op, nA0, nB0), 2048)
    oA, oB, ou = oracle.moments(op, ref)
    ea, eb = rel(nA.cpu(), oA), rel(nB.cpu(), oB)
    eu = float(np.abs(u.cpu().numpy() - ou).max() / np.abs(ou).max())
    print(f"FP64 storage after 2048 steps at 64^3: n_A {ea:.2e}, n_B {eb:.2e}, u (rel. max|u|) {eu:.2e}")
    assert ea < 1e-12 and eb < 1e-12 and eu < 1e-11
