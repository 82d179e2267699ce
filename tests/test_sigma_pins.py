"""Pins of the oracle's sigma[R] / R_s evaluator (paper section 3 and 4).

The test profiles are built to satisfy the radial mechanical equilibrium of
Eq. mech_eq_radial exactly: pick P_N(r) (a smooth step from P_in to P_out)
and set P_T = P_N + (r/2) dP_N/dr.  Then the paper's identities hold and are
checked against independent quadrature (scipy.integrate.quad) and brute-force
minimisation."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle.sigma as SG

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))

P_IN, P_OUT, R0, WIDTH = 0.3412, 0.3301, 9.3, 1.4


def PN(r):
    return P_OUT + (P_IN - P_OUT) * 0.5 * (1.0 - np.tanh((r - R0) / WIDTH))


def dPN(r):
    return -(P_IN - P_OUT) * 0.5 / WIDTH / np.cosh((r - R0) / WIDTH) ** 2


def PT(r):
    return PN(r) + 0.5 * r * dPN(r)


R_MAX = 30.0


def sigma_quad(R):
    """Eq. gen_sigma by adaptive quadrature, P_J taken literally."""
    f = lambda r: (r / R) ** 2 * ((P_IN if r < R else P_OUT) - PT(r))
    a, _ = integrate.quad(f, 0, R, epsabs=1e-13, epsrel=1e-13, limit=200)
    b, _ = integrate.quad(f, R, R_MAX, epsabs=1e-13, epsrel=1e-13, limit=200)
    return a + b


def dsigma_quad(R):
    """Eq. gen_d_sigma by adaptive quadrature."""
    f = lambda r: r * (r - R) * ((P_IN if r < R else P_OUT) - PT(r))
    a, _ = integrate.quad(f, 0, R, epsabs=1e-13, epsrel=1e-13, limit=200)
    b, _ = integrate.quad(f, R, R_MAX, epsabs=1e-13, epsrel=1e-13, limit=200)
    return -2.0 / R**3 * (a + b)


@pytest.fixture(scope="module")
def fine():
    r = np.linspace(0.0, R_MAX, 300001)
    return r, PT(r)


def test_sigma_matches_quadrature(fine):
    """The evaluator's sigma[R] (exact P_J, trapezoid P_T) equals Eq. gen_sigma by quadrature."""
    r, pt = fine
    for R in (4.0, 7.5, R0, 12.0, 20.0):
        assert SG.sigma_of_R(R, r, pt, P_IN, P_OUT) == pytest.approx(sigma_quad(R), rel=1e-7)


def test_surface_of_tension_is_the_minimum(fine):
    """R_s = argmin sigma[R] (section 3) -- closed form against brute-force
    minimisation of the quadrature, and sigma_s = dP R_s / 2 (Eq. f-statio-Rs)."""
    r, pt = fine
    res = SG.surface_of_tension(r, pt, P_IN, P_OUT)
    opt = optimize.minimize_scalar(sigma_quad, bounds=(3.0, 25.0), method="bounded",
                                   options={"xatol": 1e-9})
    assert res["Rs"] == pytest.approx(opt.x, rel=1e-5)
    assert res["sigma_s"] == pytest.approx(opt.fun, rel=1e-7)
    assert res["sigma_s"] == pytest.approx(0.5 * (P_IN - P_OUT) * res["Rs"], rel=1e-14)
    Rg, sg = SG.argmin_on_grid(r, pt, P_IN, P_OUT, 0.5 * res["Rs"], 2.0 * res["Rs"], step=0.01)
    assert Rg == pytest.approx(res["Rs"], abs=1e-4)
    assert sg == pytest.approx(res["sigma_s"], rel=1e-9)


def test_notional_derivative(fine):
    """Eq. gen_d_sigma equals d sigma[R]/dR (finite differences of the
    quadrature), vanishes at R_s, and with Eq. gen_sigma satisfies the
    generalized Laplace law Eq. LaplaceGen: dP = 2 sigma[R]/R + [d sigma/dR]."""
    r, pt = fine
    Rs = SG.surface_of_tension(r, pt, P_IN, P_OUT)["Rs"]
    for R in (5.0, 8.0, 14.0):
        h = 1e-3
        fd = (sigma_quad(R + h) - sigma_quad(R - h)) / (2 * h)
        nd = SG.notional_derivative(R, r, pt, P_IN, P_OUT)
        assert nd == pytest.approx(dsigma_quad(R), rel=1e-6, abs=1e-11)
        assert nd == pytest.approx(fd, rel=1e-5, abs=1e-10)
        lap = 2 * SG.sigma_of_R(R, r, pt, P_IN, P_OUT) / R + nd
        assert lap == pytest.approx(P_IN - P_OUT, rel=1e-6)
    assert abs(SG.notional_derivative(Rs, r, pt, P_IN, P_OUT)) < 1e-12


def test_universal_curve(fine):
    """Section 4 (Fig. 2a): sigma[R]/sigma_s = (1/3)(R_s/R)^2 + (2/3)(R/R_s)."""
    r, pt = fine
    res = SG.surface_of_tension(r, pt, P_IN, P_OUT)
    a, b = GOLD["universal_curve"]["a"], GOLD["universal_curve"]["b"]
    for x in (0.5, 0.8, 1.0, 1.3, 2.0):
        R = x * res["Rs"]
        want = a / x**2 + b * x
        assert SG.sigma_of_R(R, r, pt, P_IN, P_OUT) / res["sigma_s"] == pytest.approx(want, rel=1e-12)


def test_sharp_interface_limit():
    """A step pressure profile with a surface-tension spike of weight sigma at R0
    (mechanical equilibrium dP = 2 sigma / R0) gives R_s = R0 and sigma_s = sigma."""
    sigma = 0.01
    dP = 2 * sigma / R0
    h = 1e-4
    r = np.arange(0.0, 25.0 + h / 2, h)
    pt = np.where(r < R0, P_OUT + dP, P_OUT)
    k = int(round(R0 / h))
    pt = pt.copy()
    pt[k] -= sigma / h  # delta function of weight sigma (trapezoid: one node of weight h)
    pt[k] += 0.5 * dP  # the trapezoid half-weights of the step node
    res = SG.surface_of_tension(r, pt, P_OUT + dP, P_OUT)
    assert res["Rs"] == pytest.approx(R0, rel=1e-4)
    assert res["sigma_s"] == pytest.approx(sigma, rel=1e-4)


def test_two_dimensional_variant():
    """Two dimensions: dP_N/dr + (P_N - P_T)/r = 0 gives sigma[R] = dP R/2 + C/R,
    R_s = (2C/dP)^(1/2), sigma_s = dP R_s (checked against brute-force minimisation)."""
    r = np.linspace(0.0, R_MAX, 30001)
    pt = PN(r) + r * dPN(r)
    res = SG.surface_of_tension(r, pt, P_IN, P_OUT, dim=2)
    grid = np.linspace(4.0, 20.0, 16001)
    s = SG.sigma_of_R(grid, r, pt, P_IN, P_OUT, dim=2)
    assert res["Rs"] == pytest.approx(grid[np.argmin(s)], abs=2e-3)
    assert res["sigma_s"] == pytest.approx(s.min(), rel=1e-8)
    assert res["sigma_s"] == pytest.approx((P_IN - P_OUT) * res["Rs"], rel=1e-14)


def test_flat_sigma0():
    """Section 4: sigma_0 = int_{L/2}^{L} (P_N - P_T) dx over one interface."""
    L = 256
    z = np.arange(L)
    bump = lambda c: np.exp(-0.5 * ((z - c) / 2.0) ** 2) / (2.0 * math.sqrt(2 * math.pi))
    pn = np.full(L, 0.33)
    pt = pn - 0.07 * (bump(L / 4) + bump(3 * L / 4))
    assert SG.sigma0_flat(pn, pt) == pytest.approx(0.07, rel=1e-10)


def test_curvature_fit_recovers_coefficients():
    """Eq. sigma_c: fitting sigma(R_s) = sigma_0 (1 - 2 delta / R_s + (2kbar+k)/R_s^2)
    over A-rich (+R_s) and B-rich (-R_s) droplets recovers the coefficients."""
    s0, delta, rig = 0.104, 0.37, 1.9
    Rs = np.array([6.0, 8.0, 11.0, 16.0, 24.0, 32.0, -6.0, -9.0, -15.0, -30.0])
    sig = s0 * (1 - 2 * delta / Rs + rig / Rs**2)
    fit = SG.curvature_fit(Rs, sig)
    assert fit["sigma0"] == pytest.approx(s0, rel=1e-10)
    assert fit["delta"] == pytest.approx(delta, rel=1e-9)
    assert fit["rigidity"] == pytest.approx(rig, rel=1e-8)


def test_curvature_fit_with_fixed_sigma0():
    """Eq. sigma_c with sigma_0 held at the flat-interface value: exact data give
    back delta and 2kbar + k; a wrong sigma_0 shows up as a non-zero residual
    (the fit cannot absorb a constant offset)."""
    s0, delta, rig = 0.104, -0.21, 0.8
    Rs = np.array([5.0, 7.0, 10.0, 14.0, 20.0, 40.0, -5.0, -8.0, -13.0, -25.0])
    sig = s0 * (1 - 2 * delta / Rs + rig / Rs**2)
    fit = SG.curvature_fit(Rs, sig, sigma0=s0)
    assert fit["delta"] == pytest.approx(delta, rel=1e-10)
    assert fit["rigidity"] == pytest.approx(rig, rel=1e-9)
    lin = SG.curvature_fit(Rs, s0 * (1 - 2 * delta / Rs), order=1, sigma0=s0)
    assert lin["delta"] == pytest.approx(delta, rel=1e-12) and "rigidity" not in lin
    bad = SG.curvature_fit(Rs, sig, sigma0=1.05 * s0)
    x = 1.0 / Rs
    model = 1.05 * s0 * (1 - 2 * bad["delta"] * x + bad["rigidity"] * x**2)
    assert np.sqrt(np.mean((model - sig) ** 2)) > 1e-4
