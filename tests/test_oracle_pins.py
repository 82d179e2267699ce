"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None of them re-types the oracle's
formula: they use exact rationals, closed forms on sinusoidal fields, exact
conservation laws and symmetries, an independent NumPy transcription, and
physical consequences (demixing threshold, flat-interface mechanical
equilibrium, Laplace law)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import sc_synth as S
from oracle import np_step

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def params(orc, shape, **kw):
    return orc.Params(shape=shape, **kw)


# ------------------------------------------------------------------ stencils
@pytest.mark.parametrize("lattice,stencil", [(1, 0), (0, 0), (1, 1)])
def test_stencil_isotropy_exact(orc, lattice, stencil):
    """Section 2 after Eq. sc_force: the weights give 4th-order isotropy and
    e_2 = 1 (Eq. bulkp); the extended stencil adds 6th-order isotropy.  Checked
    in exact rationals; weights of shells 1 and 2 of D3Q19 are the printed 1/6, 1/12."""
    p = params(orc, (4, 4, 4 if lattice == 1 else 1), lattice=lattice, stencil=stencil)
    vec, W = orc.stencil(p)
    Wf = [Fraction(w).limit_denominator(1000) for w in W]
    assert all(abs(float(a) - b) < 1e-15 for a, b in zip(Wf, W))

    def mom(*powers):
        return sum(w * math.prod(int(v[m]) ** k for m, k in enumerate(powers)) for v, w in zip(vec, Wf))

    assert mom(1, 0, 0) == 0 and mom(0, 1, 0) == 0 and mom(0, 0, 1) == 0
    assert mom(2, 0, 0) == 1 == Fraction(GOLD["e2"]["value"]).limit_denominator(10)
    assert mom(0, 2, 0) == 1
    assert mom(1, 1, 0) == 0
    assert mom(4, 0, 0) == 3 * mom(2, 2, 0)
    if lattice == 1:
        assert mom(0, 0, 2) == 1 and mom(4, 0, 0) == 3 * mom(0, 2, 2)
    if stencil == 1:
        assert mom(6, 0, 0) == 15 * mom(2, 2, 2)
        assert mom(4, 2, 0) == 3 * mom(2, 2, 2)
        assert len(vec) == 32
    if lattice == 1 and stencil == 0:
        assert len(vec) == 18
        shells = sorted({int((v * v).sum()) for v in vec})
        assert shells == GOLD["forcing_shells"]["value"]
        for v, w in zip(vec, W):
            want = GOLD["W1"]["value"] if (v * v).sum() == 1 else GOLD["W2"]["value"]
            assert w == pytest.approx(want, abs=1e-16)


@pytest.mark.parametrize("lattice", [0, 1])
def test_lattice_weights_isotropy(orc, lattice):
    """Section 2: the velocity set is D3Q19 (D2Q9 in two dimensions); its
    weights satisfy sum w = 1, sum w xi xi = c_s^2 delta and the 4th-order
    moments the second-order equilibrium (Eq. feq) needs; W = w / c_s^2 gives
    the forcing weights printed after Eq. sc_force; the rest equilibrium of a
    unit field is f_i = w_i."""
    xi, w = orc.velocity_set(lattice)
    assert sorted(map(tuple, xi)) == sorted(map(tuple, np_step.velocity_set(3 if lattice == 1 else 2)[0]))
    cs2 = GOLD["cs2"]["value"]
    wf = [Fraction(x).limit_denominator(100) for x in w]
    assert sum(wf) == 1
    D = 3 if lattice == 1 else 2
    for a in range(D):
        for b in range(D):
            assert sum(x * int(v[a]) * int(v[b]) for x, v in zip(wf, xi)) == (Fraction(1, 3) if a == b else 0)
    assert sum(x * int(v[0]) ** 4 for x, v in zip(wf, xi)) == Fraction(1, 3)
    assert sum(x * int(v[0]) ** 2 * int(v[1]) ** 2 for x, v in zip(wf, xi)) == Fraction(1, 9)
    if lattice == 1:
        for v, x in zip(xi, w):
            l2 = int((v * v).sum())
            if l2:
                assert x / cs2 == pytest.approx(GOLD["W1"]["value"] if l2 == 1 else GOLD["W2"]["value"], rel=1e-15)
    shape = (3, 3, 3 if lattice == 1 else 1)
    p = params(orc, shape, lattice=lattice)
    f = orc.init(p, np.ones(p.n_sites), np.zeros(p.n_sites))
    np.testing.assert_array_equal(f[0, :, 0], w)


# ---------------------------------------------------- closed forms of Eq. sc_force / sm:pt
@pytest.mark.parametrize("stencil", [0, 1])
def test_force_on_sine_wave_closed_form(orc, stencil):
    """Eq. sc_force on n_B = a + b sin(k x) with uniform n_A: the stencil sum is
    exactly b cos(kx) S(k) with S = sin k (E4) or 14/15 sin k + 1/30 sin 2k (E6),
    so F_A^x = -G c_s^2 n_A b cos(kx) S(k), F^y = F^z = 0 (sign and prefactor)."""
    L = 16
    p = params(orc, (L, 4, 4), lattice=1, stencil=stencil, G=2.7, G_self=(0.0, 0.0))
    k = 2 * math.pi / L
    x = np.arange(L)
    a, b, nA0 = 0.6, 0.1, 0.35
    nB = np.broadcast_to(a + b * np.sin(k * x), (4, 4, L)).reshape(-1)
    nA = np.full(p.n_sites, nA0)
    FA, FB = orc.force(p, nA, nB)
    Sk = math.sin(k) if stencil == 0 else 14 / 15 * math.sin(k) + 1 / 30 * math.sin(2 * k)
    want = -p.G * GOLD["cs2"]["value"] * nA0 * b * np.cos(k * x) * Sk
    np.testing.assert_allclose(FA[0].reshape(4, 4, L)[0, 0], want, atol=1e-15)
    assert np.abs(FA[1:]).max() < 1e-15
    assert np.abs(FB).max() < 1e-15  # n_A uniform: no force on B


@pytest.mark.parametrize("stencil", [0, 1])
def test_self_force_and_pressure_tensor_closed_form(orc, stencil):
    """Eq. sm:pt on n_A = a + b sin(kx), n_B = 0, psi = n, G_AA only: with
    X(k) = sum_a W xi_x^2 cos(k xi_x) and Y(k) = sum_a W xi_y^2 cos(k xi_x),
    P^xx = c_s^2 n + G_AA c_s^2/2 n (a + b sin(kx) X(k)),
    P^yy = P^zz = c_s^2 n + G_AA c_s^2/2 n (a + b sin(kx) Y(k)), off-diagonals 0;
    and Eq. sc_force gives F^x = -G_AA c_s^2 n b cos(kx) S(k).  Counting the
    stencil's vectors by their x component: E4 X = cos k, Y = (2 + cos k)/3,
    S = sin k; E6 (shells 1-4, W = 2/15, 1/15, 1/60, 1/120) X = 14/15 cos k +
    1/15 cos 2k, Y = 3/5 + 2/5 cos k, S = 14/15 sin k + 1/30 sin 2k."""
    L = 12
    p = params(orc, (L, 5, 5), lattice=1, stencil=stencil, psi_self=0, G=0.0, G_self=(-1.3, 0.0))
    k = 2 * math.pi / L
    x = np.arange(L)
    a, b = 0.7, 0.2
    n = a + b * np.sin(k * x)
    nA = np.broadcast_to(n, (5, 5, L)).reshape(-1)
    nB = np.zeros(p.n_sites)
    if stencil == 0:
        X, Y, Sk = math.cos(k), (2 + math.cos(k)) / 3, math.sin(k)
    else:
        X = 14 / 15 * math.cos(k) + 1 / 15 * math.cos(2 * k)
        Y = 3 / 5 + 2 / 5 * math.cos(k)
        Sk = 14 / 15 * math.sin(k) + 1 / 30 * math.sin(2 * k)
    P = orc.pressure_tensor(p, nA, nB).reshape(6, 5, 5, L)[:, 0, 0]
    cs2, G = GOLD["cs2"]["value"], -1.3
    np.testing.assert_allclose(P[0], cs2 * n + 0.5 * G * cs2 * n * (a + b * np.sin(k * x) * X), atol=1e-15)
    pyy = cs2 * n + 0.5 * G * cs2 * n * (a + b * np.sin(k * x) * Y)
    np.testing.assert_allclose(P[1], pyy, atol=1e-15)
    np.testing.assert_allclose(P[2], pyy, atol=1e-15)
    assert np.abs(P[3:]).max() < 1e-15
    FA, _ = orc.force(p, nA, nB)
    np.testing.assert_allclose(FA[0].reshape(5, 5, L)[0, 0], -G * cs2 * n * b * np.cos(k * x) * Sk, atol=1e-15)


@pytest.mark.parametrize("psi_self,stencil", [(0, 0), (1, 0), (1, 1)])
def test_uniform_pressure_tensor_is_bulk_pressure(orc, psi_self, stencil):
    """Eq. bulkp (e_2 = 1): on a uniform mixture Eq. sm:pt is P delta with P the bulk pressure."""
    p = params(orc, (5, 5, 5), lattice=1, stencil=stencil, psi_self=psi_self, G=4.2, G_self=(-0.6, 0.9))
    nA0, nB0 = 0.83, 0.21
    P = orc.pressure_tensor(p, np.full(p.n_sites, nA0), np.full(p.n_sites, nB0))
    psi = (lambda n: math.exp(-1 / n)) if psi_self else (lambda n: n)
    cs2 = GOLD["cs2"]["value"]
    want = cs2 * (nA0 + nB0) + p.G * cs2 * nA0 * nB0 + 0.5 * cs2 * (-0.6 * psi(nA0) ** 2 + 0.9 * psi(nB0) ** 2)
    np.testing.assert_allclose(P[:3], want, rtol=1e-14)
    assert np.abs(P[3:]).max() < 1e-15
    assert orc.bulk_pressure(p, nA0, nB0) == pytest.approx(want, rel=1e-14)


def test_critical_self_coupling(orc):
    """Section 2 after Eq. self_p: for psi = exp(-1/n) the critical self coupling
    is G_c c_s^2 ~ -2.463.  With G_AA = G_c the bulk pressure of Eq. bulkp has
    dP/dn = d2P/dn2 = 0 at the critical density (n = 1), and G_c = -e^2."""
    Gc = -math.e**2
    assert Gc * GOLD["cs2"]["value"] == pytest.approx(GOLD["Gc_cs2"]["value"], abs=5e-4)
    p = params(orc, (1, 1, 1), lattice=1, psi_self=1, G_self=(Gc, 0.0))
    P = lambda n: orc.bulk_pressure(p, n, 1e-300)
    h = 1e-3
    d1 = (P(1 + h) - P(1 - h)) / (2 * h)
    d2 = (P(1 + h) - 2 * P(1) + P(1 - h)) / h**2
    assert abs(d1) < 1e-6 and abs(d2) < 1e-5
    pp = params(orc, (1, 1, 1), lattice=1, psi_self=1, G_self=(0.95 * Gc, 0.0))
    assert min((orc.bulk_pressure(pp, n + h, 0) - orc.bulk_pressure(pp, n - h, 0)) for n in np.linspace(0.5, 2, 31)) > 0


# --------------------------------------------------------------- brute force
@pytest.mark.parametrize("dim,stencil,psi_self", [(3, 0, 1), (3, 1, 1), (2, 0, 0), (3, 0, 0)])
def test_c_oracle_matches_numpy_transcription(orc, dim, stencil, psi_self):
    """The C oracle and the independent NumPy (np.roll) transcription agree to
    round-off after 10 steps on tiny lattices, with unequal tau and asymmetric G."""
    shape = (5, 6, 7) if dim == 3 else (1, 8, 9)
    nA, nB = S.droplet(shape, (3, 3, 2 if dim == 3 else 0), 2.0, n_in=0.8, n_out=0.2, amplitude=1e-2)
    p = params(orc, shape[::-1], lattice=1 if dim == 3 else 0, stencil=stencil, psi_self=psi_self,
               tau=(1.0, 0.9), G=2.5, G_self=(-0.6, 0.3))
    f = orc.step(p, orc.init(p, nA, nB), 10)
    a, b, u = orc.moments(p, f)
    g = np_step.init(nA, nB, dim)
    for _ in range(10):
        g = np_step.step(g, dim, p.tau, p.G, p.G_self, bool(psi_self), bool(stencil))
    a2, b2, u2 = np_step.moments(g, dim, p.G, p.G_self, bool(psi_self), bool(stencil))
    assert np.abs(a - a2.ravel()).max() < 1e-13
    assert np.abs(b - b2.ravel()).max() < 1e-13
    assert np.abs(u - u2.reshape(3, -1)).max() < 1e-13


def test_step_sites_matches_full_step(orc):
    """The per-site one-step evaluation agrees with a full step at those sites."""
    shape = (6, 5, 4)
    nA, nB = S.droplet(shape, (2, 2, 3), 1.5, n_in=0.8, n_out=0.2, amplitude=1e-2)
    p = params(orc, shape[::-1], lattice=1, psi_self=1, tau=(1.0, 0.7), G=2.5, G_self=(-0.4, 0.0))
    f = orc.step(p, orc.init(p, nA, nB), 3)
    full = orc.step(p, f, 1)
    sel = np.array([0, 7, 33, p.n_sites - 1])
    part = orc.step_sites(p, f, sel)
    np.testing.assert_array_equal(part, full[:, :, sel])


# ------------------------------------------------------------- invariants
def test_mass_conservation(orc):
    """Eq. lbm: streaming permutes populations and sum_i Omega_i = sum_i F_i = 0,
    so each component's mass is conserved exactly (round-off only)."""
    shape = (12, 12, 12)
    nA, nB = S.droplet(shape, (6, 6, 6), 4.0, n_in=0.85, n_out=0.15)
    p = params(orc, shape[::-1], lattice=1, psi_self=1, tau=(1.0, 0.8), G=2.5, G_self=(-0.6, 0.0))
    f = orc.init(p, nA, nB)
    m0, _ = orc.totals(p, f)
    g = orc.step(p, f, 50)
    assert np.isfinite(g).all()
    m1, _ = orc.totals(p, g)
    np.testing.assert_allclose(m1, m0, rtol=1e-13)
    assert m0 == pytest.approx([nA.sum(), nB.sum()], rel=1e-13)


@pytest.mark.parametrize("G_self", [(0.0, 0.0), (-0.6, 0.4)])
def test_momentum_conservation_equal_tau(orc, G_self):
    """With tau_A = tau_B the collision adds exactly F(x) per site (Eq. u with
    Eqs. omega_i and Guo), and sum_x F vanishes on a periodic lattice (pairs of
    Eq. sc_force cancel), so total momentum is conserved for any G."""
    shape = (10, 11, 12)
    nA, nB = S.droplet(shape, (5, 5, 6), 3.5, n_in=0.85, n_out=0.15, amplitude=1e-2)
    p = params(orc, shape[::-1], lattice=1, psi_self=1, tau=(0.8, 0.8), G=2.5, G_self=G_self)
    f = orc.step(p, orc.init(p, nA, nB), 40)
    assert np.isfinite(f).all()
    _, mom = orc.totals(p, f)
    assert np.abs(mom).max() < 1e-12


def test_swap_symmetry_bitwise(orc):
    """Section 2 (remarks after Eq. sc_force): with G_AA = G_BB (and tau_A =
    tau_B) the dynamics is invariant under A <-> B; swapping the initial fields
    swaps every field bit for bit."""
    shape = (9, 8, 7)
    nA, nB = S.droplet(shape, (4, 4, 3), 2.5, n_in=0.85, n_out=0.15, amplitude=1e-2)
    p = params(orc, shape[::-1], lattice=1, psi_self=1, tau=(0.9, 0.9), G=2.5, G_self=(-0.5, -0.5))
    f = orc.step(p, orc.init(p, nA, nB), 20)
    g = orc.step(p, orc.init(p, nB, nA), 20)
    assert np.isfinite(f).all()
    np.testing.assert_array_equal(f[0], g[1])
    np.testing.assert_array_equal(f[1], g[0])


def test_uniform_mixture_is_stationary_bitwise(orc):
    """Eq. sc_force on a uniform mixture: every +/- pair cancels, so F = 0 and
    u = 0 exactly; every site then runs the same arithmetic, so the field stays
    uniform bit for bit, and at the rest equilibrium to round-off (the only
    round-off is in n = sum_i f_i)."""
    p = params(orc, (6, 7, 8), lattice=1, psi_self=1, tau=(0.7, 1.3), G=4.2, G_self=(-0.6, 0.2))
    nA, nB = S.uniform((8, 7, 6), 0.37, 0.71)
    f0 = orc.init(p, nA, nB)
    FA, FB = orc.force(p, nA, nB)
    assert not FA.any() and not FB.any()
    f = orc.step(p, f0, 25)
    _, _, u = orc.moments(p, f)
    assert not u.any()
    assert not np.ptp(f, axis=2).any()
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau,G_self", [(1.0, (0.0, 0.0)), (0.8, (-0.6, 0.0))])
def test_flat_interface_normal_pressure_constant(orc, tau, G_self):
    """Section 2 after Eq. sm:pt: at a converged flat interface the normal
    component of the lattice pressure tensor is constant to machine precision
    (nearest-neighbour stencil), so P_N(z) has no interface structure while
    P_T(z) does."""
    Lz = 48
    nA, nB = S.slab((Lz, 1, 1), 24, 0.95, 0.05)
    p = params(orc, (1, 1, Lz), lattice=1, psi_self=1, tau=(tau, tau), G=4.2, G_self=G_self)
    f = orc.step(p, orc.init(p, nA, nB), 25000)
    a, b, u = orc.moments(p, f)
    prof = orc.profile(p, a, b, orc.PLANAR_Z, nbins=Lz)
    PN, PT = prof[:, 1], prof[:, 2]
    assert np.abs(u).max() < 1e-13
    assert np.ptp(PN) < 1e-13
    assert np.ptp(PT) > 1e-2


# --------------------------------------------------------- physical checks
def _variance_after(orc, G, steps):
    shape = (1, 64, 64)
    nA, nB = S.droplet(shape, (32, 32, 0), 12.0)
    p = params(orc, (64, 64, 1), lattice=0, psi_self=0, G=G)
    a, _, _ = orc.moments(p, orc.step(p, orc.init(p, nA, nB), steps), with_u=False)
    return nA.var(), a.var()


def test_demixing_threshold_and_coupling_units(orc):
    """Eq. bulkp with psi = n: f = c_s^2 sum n ln n + G c_s^2 n_A n_B is convex
    along (1, -1) at n_A = n_B = n/2 iff G n < 2.  A droplet at total density 1
    therefore dissolves for G = 1.4 and persists for G = 4.2 = 1.4 / c_s^2, the
    reading of a coupling quoted as G c_s^2 (section 4 quotes G c_s^2)."""
    v0, v_low = _variance_after(orc, 1.4, 1500)
    _, v_high = _variance_after(orc, 4.2, 1500)
    assert v_low < 0.05 * v0
    assert v_high > 0.9 * v0


def test_laplace_law_two_dimensions(orc):
    """Eq. f-statio-Rs / Eq. LaplaceGen in two dimensions: dP R_s approaches the
    flat-interface tension sigma_0 (section 4) as the droplet grows."""
    import oracle.sigma as SG

    G = 4.2
    Ly = 96
    nA, nB = S.slab((1, Ly, 1), 48, 0.95, 0.05, axis="y")
    p = params(orc, (1, Ly, 1), lattice=0, psi_self=0, G=G)
    a, b, _ = orc.moments(p, orc.step(p, orc.init(p, nA, nB), 15000), with_u=False)
    P = orc.pressure_tensor(p, a, b)
    sig0 = SG.sigma0_flat(P[1], P[0])
    nin, nout = a.max(), a.min()
    ratios = []
    for L, R in ((40, 8), (80, 17)):
        nA, nB = S.droplet((1, L, L), (L // 2, L // 2, 0), R, n_in=nin, n_out=nout, amplitude=0)
        p = params(orc, (L, L, 1), lattice=0, psi_self=0, G=G)
        a, b, _ = orc.moments(p, orc.step(p, orc.init(p, nA, nB), 5000), with_u=False)
        rows = orc.profile(p, a, b, orc.RADIAL, centre=(L // 2, L // 2, 0), bin_width=0.5, nbins=L)
        r, _, PT, _, _ = SG.clean_profile(rows)
        c = L // 2 + L * (L // 2)
        res = SG.surface_of_tension(r, PT, orc.bulk_pressure(p, a[c], b[c]), orc.bulk_pressure(p, a[-1], b[-1]),
                                    dim=2)
        assert abs(res["Rs"] - R) < 2.0
        ratios.append(res["sigma_s"] / sig0)
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1)
    assert abs(ratios[1] - 1) < 0.08


def test_profile_radial_bins_brute_force(orc):
    """Radial binning (section 3 decomposition, 0.5 lu shells): per-bin site
    counts and mean radii equal a brute-force count; on a uniform field every
    bin carries P_N = P_T = bulk pressure."""
    shape = (10, 10, 10)
    p = params(orc, shape[::-1], lattice=1, psi_self=1, G=4.2, G_self=(-0.3, 0.0))
    nA, nB = S.uniform(shape, 0.6, 0.3)
    rows = orc.profile(p, nA, nB, orc.RADIAL, centre=(5, 5, 5), bin_width=0.5, nbins=20)
    r = S.min_image_radius(shape, (5, 5, 5)).ravel()
    k = np.floor(r / 0.5).astype(int)
    for b in range(20):
        m = k == b
        assert rows[b, 5] == m.sum()
        if m.any():
            assert rows[b, 0] == pytest.approx(r[m].mean(), rel=1e-14)
            assert rows[b, 1] == pytest.approx(orc.bulk_pressure(p, 0.6, 0.3), rel=1e-14)
            assert rows[b, 2] == pytest.approx(orc.bulk_pressure(p, 0.6, 0.3), rel=1e-14)
        else:
            assert not rows[b].any()


# ------------------------------------- off-diagonal pressure tensor and the profile projections
def _diagonal_wave(L, k, a, b, axes):
    """psi = n_A = a + b sin(theta), theta = k * (sum of the listed coordinates), on an L^3 box
    (site order x fastest); returns (n_A as [L, L, L] indexed [z, y, x], theta)."""
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    coord = {"x": x, "y": y, "z": z}
    theta = k * sum(coord[c] for c in axes)
    return a + b * np.sin(theta), theta


def test_pressure_tensor_off_diagonal_closed_form(orc):
    """Eq. sm:pt with psi = n, G_AA only, nearest-neighbour stencil (W = 1/6, 1/12), on a wave
    along the body diagonal, n = a + b sin(theta), theta = k (x + y + z).  Counting the 18
    vectors: only the four xi = (+-1, +-1, 0) weigh xi_x xi_y; (1, 1, 0) and (-1, -1, 0) see
    theta +- 2k, (1, -1, 0) and (-1, 1, 0) see theta, so sum_a W xi_x xi_y n(x + xi_a) =
    (b / 6) sin(theta) (cos 2k - 1), and by symmetry the same for xz and yz.  Each diagonal
    collects 2 vectors at theta +- k (W = 1/6) and 8 at theta +- 2k, theta (W = 1/12):
    sum_a W xi_x^2 n(x + xi_a) = a + b sin(theta) (1 + cos k + cos 2k) / 3.  So
    P^mumu = c_s^2 n + G c_s^2/2 n (a + b sin(theta) (1 + cos k + cos 2k)/3) and
    P^munu = G c_s^2/2 n (b / 6) sin(theta) (cos 2k - 1) for mu != nu."""
    L = 12
    k = 2 * math.pi / L
    a, b, G = 0.7, 0.2, -1.3
    n, th = _diagonal_wave(L, k, a, b, "xyz")
    p = params(orc, (L, L, L), lattice=1, stencil=0, psi_self=0, G=0.0, G_self=(G, 0.0))
    P = orc.pressure_tensor(p, n.ravel(), np.zeros(L**3)).reshape(6, L, L, L)
    cs2 = GOLD["cs2"]["value"]
    diag = cs2 * n + 0.5 * G * cs2 * n * (a + b * np.sin(th) * (1 + math.cos(k) + math.cos(2 * k)) / 3)
    off = 0.5 * G * cs2 * n * (b / 6) * np.sin(th) * (math.cos(2 * k) - 1)
    assert np.abs(off).max() > 1e-3  # the off-diagonals are far from zero here
    for c in range(3):
        np.testing.assert_allclose(P[c], diag, atol=1e-15)
    for c in range(3, 6):
        np.testing.assert_allclose(P[c], off, atol=1e-15)


def test_pressure_tensor_planar_diagonal_wave_closed_form(orc):
    """As above with theta = k (x + y): P^xy = G c_s^2/2 n (b/6) sin(theta)(cos 2k - 1),
    P^xz = P^yz = 0 (the (+-1, 0, +-1) vectors cancel in pairs), P^xx = P^yy with
    sum_a W xi_x^2 n(x + xi_a) = a + b sin(theta) ((2/3) cos k + (1/6) cos 2k + 1/6) and
    P^zz with sum_a W xi_z^2 n(x + xi_a) = a + b sin(theta) (1/3 + (2/3) cos k)."""
    L = 12
    k = 2 * math.pi / L
    a, b, G = 0.6, 0.25, 0.9
    n, th = _diagonal_wave(L, k, a, b, "xy")
    p = params(orc, (L, L, L), lattice=1, stencil=0, psi_self=0, G=0.0, G_self=(G, 0.0))
    P = orc.pressure_tensor(p, n.ravel(), np.zeros(L**3)).reshape(6, L, L, L)
    cs2 = GOLD["cs2"]["value"]
    s = np.sin(th)
    pxx = cs2 * n + 0.5 * G * cs2 * n * (a + b * s * (2 / 3 * math.cos(k) + math.cos(2 * k) / 6 + 1 / 6))
    pzz = cs2 * n + 0.5 * G * cs2 * n * (a + b * s * (1 / 3 + 2 / 3 * math.cos(k)))
    pxy = 0.5 * G * cs2 * n * (b / 6) * s * (math.cos(2 * k) - 1)
    np.testing.assert_allclose(P[0], pxx, atol=1e-15)
    np.testing.assert_allclose(P[1], pxx, atol=1e-15)
    np.testing.assert_allclose(P[2], pzz, atol=1e-15)
    np.testing.assert_allclose(P[3], pxy, atol=1e-15)
    assert np.abs(P[4:]).max() < 1e-15


def _min_image_displacement(shape_zyx, centre):
    """(dx, dy, dz) [3, N] from centre (x, y, z) to every site, each in [-L/2, L/2) by
    brute force over the periodic images -L, 0, +L."""
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for c, L, ce in ((x, nx, centre[0]), (y, ny, centre[1]), (z, nz, centre[2])):
        cand = np.stack([c - ce - L, c - ce, c - ce + L]).astype(float)
        ok = (cand >= -L / 2) & (cand < L / 2)
        out.append((cand * ok).sum(0).ravel())
    return np.array(out)


def _radial_brute_force(shape_zyx, centre, bin_width, nbins, Pfull, nA, nB):
    """Section 3's decomposition done site by site: r from the minimum image, the unit vector
    rhat, P_N = rhat . P . rhat with the full symmetric 3 x 3 matrix, P_T = (tr P - P_N) / 2
    (tr P / 3 for both at r = 0), then per-bin means of (r, P_N, P_T, n_A, n_B) and counts.
    Pfull: [3, 3, N]."""
    d = _min_image_displacement(shape_zyx, centre)  # [3, N] as (dx, dy, dz)
    r = np.sqrt((d**2).sum(0))
    with np.errstate(invalid="ignore", divide="ignore"):
        e = np.where(r > 0, d / r, 0.0)
    tr = Pfull[0, 0] + Pfull[1, 1] + Pfull[2, 2]
    PN = np.einsum("ms,mns,ns->s", e, Pfull, e)
    PN = np.where(r > 0, PN, tr / 3)
    PT = np.where(r > 0, (tr - PN) / 2, tr / 3)
    kbin = np.floor(r / bin_width).astype(int)
    keep = kbin < nbins
    out = np.zeros((nbins, 6))
    cnt = np.bincount(kbin[keep], minlength=nbins)[:nbins]
    for c, v in enumerate((r, PN, PT, nA, nB)):
        s = np.bincount(kbin[keep], weights=v[keep], minlength=nbins)[:nbins]
        out[:, c] = np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)
    out[:, 5] = cnt
    return out


def _full_matrix(P6):
    """[6, N] (xx, yy, zz, xy, xz, yz) -> [3, 3, N]."""
    xx, yy, zz, xy, xz, yz = P6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def test_radial_profile_projection_on_closed_form_tensor(orc):
    """Eq. pt_projection on the body-diagonal wave, where the off-diagonal components are of
    the same order as the anisotropic part of the diagonal: the oracle's radial rows equal the
    brute-force projection rhat . P . rhat of the closed-form tensor (no oracle tensor used),
    binned by hand.  A dropped factor 2 on the off-diagonal terms moves P_N by
    sum_{mu != nu} rhat_mu rhat_nu P^munu / 2, several times the tolerance."""
    L = 12
    k = 2 * math.pi / L
    a, b, G = 0.7, 0.2, -1.3
    n, th = _diagonal_wave(L, k, a, b, "xyz")
    cs2 = GOLD["cs2"]["value"]
    diag = (cs2 * n + 0.5 * G * cs2 * n * (a + b * np.sin(th) * (1 + math.cos(k) + math.cos(2 * k)) / 3)).ravel()
    off = (0.5 * G * cs2 * n * (b / 6) * np.sin(th) * (math.cos(2 * k) - 1)).ravel()
    P6 = np.array([diag, diag, diag, off, off, off])
    centre = (5.0, 4.0, 7.0)
    p = params(orc, (L, L, L), lattice=1, stencil=0, psi_self=0, G=0.0, G_self=(G, 0.0))
    rows = orc.profile(p, n.ravel(), np.zeros(L**3), orc.RADIAL, centre=centre, bin_width=0.5, nbins=24)
    want = _radial_brute_force((L, L, L), centre, 0.5, 24, _full_matrix(P6), n.ravel(), np.zeros(L**3))
    np.testing.assert_array_equal(rows[:, 5], want[:, 5])
    np.testing.assert_allclose(rows[:, :5], want[:, :5], rtol=0, atol=1e-14)
    # the off-diagonal share of P_N is resolved: halving it would move some bin by far more than 1e-14
    half = _radial_brute_force((L, L, L), centre, 0.5, 24, _full_matrix(P6 * np.array([1, 1, 1, .5, .5, .5])[:, None]),
                               n.ravel(), np.zeros(L**3))
    assert np.abs(half[:, 1] - want[:, 1]).max() > 1e-4


def test_radial_profile_projection_on_droplet(orc):
    """Eq. pt_projection on a non-uniform, off-centre, noisy two-component droplet with both
    couplings and psi = exp(-1/n): every radial row (count, mean r, P_N, P_T, n_A, n_B) equals
    the brute-force projection of the pinned Eq. sm:pt tensor with the full 3 x 3 matrix, and
    P_T is (tr P - P_N) / 2 bin by bin (the trace binned on its own)."""
    shape = (14, 13, 12)  # (nz, ny, nx)
    nA, nB = S.droplet(shape, (5, 7, 6), 3.5, n_in=0.85, n_out=0.15, amplitude=2e-2)
    p = params(orc, shape[::-1], lattice=1, stencil=0, psi_self=1, G=2.5, G_self=(-0.6, 0.3))
    f = orc.step(p, orc.init(p, nA, nB), 20)
    a, bB, _ = orc.moments(p, f, with_u=False)
    P6 = orc.pressure_tensor(p, a, bB)
    assert np.abs(P6[3:]).max() > 1e-3
    centre = (6.0, 7.0, 5.0)
    rows = orc.profile(p, a, bB, orc.RADIAL, centre=centre, bin_width=0.5, nbins=20)
    want = _radial_brute_force(shape, centre, 0.5, 20, _full_matrix(P6), a, bB)
    np.testing.assert_array_equal(rows[:, 5], want[:, 5])
    np.testing.assert_allclose(rows[:, :5], want[:, :5], rtol=0, atol=1e-14)
    tr = P6[0] + P6[1] + P6[2]
    d = _min_image_displacement(shape, centre)
    r = np.sqrt((d**2).sum(0))
    kb = np.floor(r / 0.5).astype(int)
    m = kb < 20
    trbin = np.bincount(kb[m], weights=tr[m], minlength=20)[:20] / np.maximum(rows[:, 5], 1)
    nz = rows[:, 5] > 0
    np.testing.assert_allclose(rows[nz, 2], (trbin[nz] - rows[nz, 1]) / 2, rtol=0, atol=1e-14)


def test_axis_profile_is_section3_line(orc):
    """Section 3's estimator along the x axis through the centre node: row k is the site
    (c_x + k, c_y, c_z) with coordinate k, P_N = P^xx, P_T = P^yy, its densities and count 1.
    On the x wave of the closed-form test (P^xx and P^yy differ there) the rows equal the closed
    forms; on a noisy off-centre droplet they equal the pinned tensor at those sites."""
    L = 12
    k = 2 * math.pi / L
    a, b, G = 0.7, 0.2, -1.3
    p = params(orc, (L, 5, 5), lattice=1, stencil=0, psi_self=0, G=0.0, G_self=(G, 0.0))
    x = np.arange(L)
    n = a + b * np.sin(k * x)
    nA = np.broadcast_to(n, (5, 5, L)).reshape(-1)
    cs2 = GOLD["cs2"]["value"]
    pxx = cs2 * n + 0.5 * G * cs2 * n * (a + b * np.sin(k * x) * math.cos(k))
    pyy = cs2 * n + 0.5 * G * cs2 * n * (a + b * np.sin(k * x) * (2 + math.cos(k)) / 3)
    cx = 3
    rows = orc.profile(p, nA, np.zeros(p.n_sites), orc.AXIS_X, centre=(cx, 2, 1), nbins=L - cx)
    xs = cx + np.arange(L - cx)
    np.testing.assert_array_equal(rows[:, 0], np.arange(L - cx))
    np.testing.assert_allclose(rows[:, 1], pxx[xs], atol=1e-15)
    np.testing.assert_allclose(rows[:, 2], pyy[xs], atol=1e-15)
    np.testing.assert_allclose(rows[:, 3], n[xs], atol=1e-15)
    assert not rows[:, 4].any() and (rows[:, 5] == 1).all()

    shape = (9, 10, 16)  # (nz, ny, nx)
    nA, nB = S.droplet(shape, (4, 5, 8), 3.0, n_in=0.85, n_out=0.15, amplitude=2e-2)
    p = params(orc, shape[::-1], lattice=1, stencil=0, psi_self=1, G=2.5, G_self=(-0.6, 0.3))
    P6 = orc.pressure_tensor(p, nA, nB).reshape(6, *shape)
    c = (7, 4, 3)  # (x, y, z), not the droplet's centre
    rows = orc.profile(p, nA, nB, orc.AXIS_X, centre=c, nbins=16 - c[0])
    xs = c[0] + np.arange(16 - c[0])
    np.testing.assert_array_equal(rows[:, 1], P6[0, c[2], c[1], xs])
    np.testing.assert_array_equal(rows[:, 2], P6[1, c[2], c[1], xs])
    np.testing.assert_array_equal(rows[:, 3], nA.reshape(shape)[c[2], c[1], xs])
    np.testing.assert_array_equal(rows[:, 4], nB.reshape(shape)[c[2], c[1], xs])
    assert np.abs(P6[0, c[2], c[1], xs] - P6[1, c[2], c[1], xs]).max() > 1e-3
