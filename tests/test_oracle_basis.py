"""Pins for the basis functions and the regression rows (Sec. III-A, III-B).

Wendland C2 is identified by the properties that define it, not by retyping
its formula; the Gaussian regression row is pinned by numerical quadrature of
the conditional expectation that defines it (Sec. III-B).
"""
import math

import numpy as np
import pytest

from oracle import rbf_oracle as O


@pytest.mark.parametrize("rho", [0.3, 0.6, 1.7])
def test_wendland_defining_properties(rho):
    f = lambda r: O.phi(r, O.WENDLAND, rho=rho)
    assert f(0.0) == pytest.approx(1.0, abs=1e-15)
    # compact support
    assert np.all(f(np.array([rho, 1.01 * rho, 3 * rho])) == 0.0)
    # a degree-5 polynomial on [0, rho]
    s = np.linspace(0, rho, 40)
    coef = np.polyfit(s, f(s), 5)
    assert np.max(np.abs(np.polyval(coef, s) - f(s))) < 1e-12
    # fourfold root at r = rho: phi / (1 - r/rho)^4 is affine in r
    s2 = np.linspace(0.05, 0.9, 20) * rho
    ratio = f(s2) / (1 - s2 / rho) ** 4
    lin = np.polyfit(s2, ratio, 1)
    assert np.max(np.abs(np.polyval(lin, s2) - ratio)) < 1e-10
    # smooth (even) at the origin: phi'(0) = 0 by one-sided difference
    e = 1e-6 * rho
    assert abs((f(e) - f(0.0)) / e) < 1e-4
    # C2 at the support edge: one-sided first and second differences vanish
    e = 1e-4 * rho
    d1 = (f(rho) - f(rho - e)) / e
    d2 = (f(rho) - 2 * f(rho - e) + f(rho - 2 * e)) / e ** 2
    assert abs(d1) < 1e-6 and abs(d2) < 1e-3


def test_wendland_positive_definite_in_plane():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1.0, (60, 2))
    r = np.linalg.norm(x[:, None] - x[None], axis=2)
    G = O.phi(r, O.WENDLAND, rho=0.5)
    assert np.linalg.eigvalsh(G).min() > 0


@pytest.mark.parametrize("kind", [O.WENDLAND, O.GAUSSIAN])
def test_grad_coef_matches_finite_difference(kind):
    rng = np.random.default_rng(1)
    rho, sigma = 0.6, 0.11
    c = np.array([0.3, -0.2])
    for _ in range(50):
        x = c + rng.uniform(-0.5, 0.5, 2)
        r = np.linalg.norm(x - c)
        g = O.grad_coef(r, kind, rho, sigma) * (x - c)
        e = 1e-6
        fd = np.zeros(2)
        for k in range(2):
            xp = x.copy(); xm = x.copy(); xp[k] += e; xm[k] -= e
            fd[k] = (O.phi(np.linalg.norm(xp - c), kind, rho, sigma)
                     - O.phi(np.linalg.norm(xm - c), kind, rho, sigma)) / (2 * e)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_gaussian_moment_row_equals_conditional_expectation():
    """m(x) = E[k_sigma(xbar; c) | x] with xbar ~ N(x, s_eps^2 I) (Sec. III-B),
    by 2-D Gauss-Hermite quadrature; must equal (s^2/st^2) k_st(x; c)."""
    sigma, eps = 0.04, 0.1
    gx, gw = np.polynomial.hermite_e.hermegauss(80)   # weight exp(-t^2/2)
    gw = gw / math.sqrt(2 * math.pi)
    rng = np.random.default_rng(0)
    c = np.array([[0.0, 0.0]])
    for _ in range(10):
        x = rng.uniform(-0.15, 0.15, 2)
        X = x[0] + eps * gx[:, None]
        Y = x[1] + eps * gx[None, :]
        val = np.exp(-((X - c[0, 0]) ** 2 + (Y - c[0, 1]) ** 2) / (2 * sigma ** 2))
        quad = float(gw @ val @ gw)
        row = O.design_rows(x[None, :], c, O.GAUSSIAN, sigma=sigma, cutoff_mult=50.0,
                            noise=eps)[0, 0]
        assert row == pytest.approx(quad, rel=1e-9, abs=1e-14)


def test_wendland_row_is_phi_and_noise_is_unused():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (7, 2)); c = rng.uniform(0, 1, (5, 2))
    a = O.design_rows(x, c, O.WENDLAND, rho=0.6, noise=0.0)
    b = O.design_rows(x, c, O.WENDLAND, rho=0.6, noise=0.3)
    r = np.linalg.norm(x[:, None] - c[None], axis=2)
    assert np.array_equal(a, b)
    assert np.allclose(a, O.phi(r, O.WENDLAND, rho=0.6))


def _golden_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "basis_closed_form.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            yield line.split()


def test_basis_matches_closed_form_fixture():
    """Hand-derived values of phi, its gradient coefficient and the Gaussian
    regression-row scale (tests/golden/basis_closed_form.txt)."""
    rows = list(_golden_rows())
    assert len(rows) == 9
    for kind, r, par, noise, ph, g, row in rows:
        kind, r, par = int(kind), float(r), float(par)
        kw = dict(rho=par) if kind == O.WENDLAND else dict(sigma=par)
        if ph != "-":
            assert O.phi(r, kind, **kw) == pytest.approx(float(ph), rel=1e-13, abs=1e-15)
            assert O.grad_coef(r, kind, **kw) == pytest.approx(float(g), rel=1e-13, abs=1e-15)
        if row != "-":
            m = O.design_rows(np.array([[r, 0.0]]), np.zeros((1, 2)), kind, sigma=par, noise=float(noise))
            assert m[0, 0] == pytest.approx(float(row), rel=1e-13)
