"""Pins of the oracle's regularized Stokeslet and stresslet (the paper names
them as future work and gives no kernel; the blob is that of Cortez, Fauci
and Medovikov, 2005).  Each test checks the oracle against something other
than itself:

* the kernels: at eps = 0 they are eqs. (1.2a,b); the regularized Stokeslet
  flow u = S^eps g is divergence-free and solves the blob-forced Stokes
  equations lap u - grad p = -15 eps^4 s^(-7/2) g with the pressure
  p = (g.d)(2 r^2 + 5 eps^2) s^(-5/2) (checked by central differences); the
  stresslet is -1/6 of that flow's stress -p delta + grad u + grad u^T;
* the coefficient recurrence for (|x - y|^2 + eps^2)^(-nu): the Gegenbauer
  generating function (scipy);
* the Taylor coefficients of the kernels: a power-series expansion of the
  kernels in t (tests/jet.py);
* the far field: geometric convergence to the direct sum in p;
* the treecode: theta -> 0 gives the regularized direct sum, eps -> 0 the
  treecode of eqs. (1.2a,b).
"""
import numpy as np
import pytest
from scipy.special import eval_gegenbauer

import oracle
from paper_1811_12498_gb300 import inputs
from tests.jet import reg_kernel_jets


def _rng(s):
    return np.random.default_rng(5000 + s)


def test_regularized_kernels_reduce_to_eqs_1_2_at_eps_zero():
    rng = _rng(1)
    for _ in range(5):
        x, y = rng.standard_normal(3), rng.standard_normal(3)
        np.testing.assert_allclose(oracle.stokeslet_reg(x, y, 0.0), oracle.stokeslet(x, y), rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(oracle.stresslet_reg(x, y, 0.0), oracle.stresslet(x, y), rtol=1e-14, atol=1e-15)


def _u(x, y, eps, g):
    return oracle.stokeslet_reg(x, y, eps) @ g


def _grad_u(x, y, eps, g, h):
    """J[i, k] = d u_k / d x_i by central differences."""
    J = np.empty((3, 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        J[i] = (_u(x + e, y, eps, g) - _u(x - e, y, eps, g)) / (2 * h)
    return J


@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0])
def test_regularized_stokeslet_solves_the_blob_forced_stokes_equations(eps):
    rng = _rng(2)
    h = 1e-3 * eps
    for _ in range(4):
        y = rng.standard_normal(3)
        x = y + rng.standard_normal(3) * eps
        g = rng.standard_normal(3)
        d = x - y
        r2 = d @ d
        s = r2 + eps * eps
        # divergence
        assert abs(np.trace(_grad_u(x, y, eps, g, h))) <= 1e-6 * np.linalg.norm(_u(x, y, eps, g)) / eps
        # lap u - grad p + blob g = 0
        lap = np.zeros(3)
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            lap += (_u(x + e, y, eps, g) - 2 * _u(x, y, eps, g) + _u(x - e, y, eps, g)) / h ** 2

        def pres(xx):
            dd = xx - y
            ss = dd @ dd + eps * eps
            return (g @ dd) * (2 * (dd @ dd) + 5 * eps * eps) / ss ** 2.5

        gp = np.array([(pres(x + np.eye(3)[i] * h) - pres(x - np.eye(3)[i] * h)) / (2 * h) for i in range(3)])
        blob = 15 * eps ** 4 / s ** 3.5 * g
        scale = np.linalg.norm(lap) + np.linalg.norm(gp) + np.linalg.norm(blob)
        np.testing.assert_allclose(lap - gp + blob, 0.0, atol=1e-5 * scale)


@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0])
def test_regularized_stresslet_is_minus_one_sixth_of_the_stokeslet_stress(eps):
    """sigma_ik of the flow of a regularized point force along e_j equals
    -6 T^eps_ijk (the singular pair: the stress of the Stokeslet of eq. (1.2a)
    is -6 times eq. (1.2b))."""
    rng = _rng(3)
    h = 1e-4 * eps
    for _ in range(3):
        y = rng.standard_normal(3)
        x = y + rng.standard_normal(3) * eps
        d = x - y
        s = d @ d + eps * eps
        T = oracle.stresslet_reg(x, y, eps)
        for j in range(3):
            g = np.eye(3)[j]
            p = (g @ d) * (2 * (d @ d) + 5 * eps * eps) / s ** 2.5
            J = _grad_u(x, y, eps, g, h)
            sigma = -p * np.eye(3) + J + J.T
            np.testing.assert_allclose(sigma, -6 * T[:, j, :], rtol=1e-6, atol=1e-6 * np.abs(sigma).max())


@pytest.mark.parametrize("two_nu", [1, 3, 5])
def test_coefficient_recurrence_matches_gegenbauer_generating_function(two_nu):
    """(R_e^2 - 2 tau d.u + tau^2)^(-nu) = sum_n C_n^nu(d.u / R_e) tau^n / R_e^(2 nu + n),
    R_e^2 = |d|^2 + eps^2: the coefficients of level n summed against u^k
    give R_e^(-2nu-n) C_n^nu(d.u / R_e)."""
    rng = _rng(4 + two_nu)
    P = 10
    nu = two_nu / 2.0
    for eps in (0.0, 0.4, 2.0):
        d = rng.standard_normal(3) * 1.5
        c = oracle.coeffs_nu(d, eps, two_nu, P)
        Re = np.sqrt(d @ d + eps * eps)
        for _ in range(3):
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            for n in range(P + 1):
                s = sum(c[k1, k2, n - k1 - k2] * u[0] ** k1 * u[1] ** k2 * u[2] ** (n - k1 - k2)
                        for k1 in range(n + 1) for k2 in range(n - k1 + 1))
                ref = eval_gegenbauer(n, nu, (d @ u) / Re) / Re ** (2 * nu + n)
                assert abs(s - ref) <= 1e-12 * max(1.0, abs(ref)) * Re ** (-2 * nu - n), (eps, n, s, ref)


@pytest.mark.parametrize("p", [0, 2, 5])
@pytest.mark.parametrize("eps", [0.1, 0.7])
def test_regularized_taylor_coefficients_match_power_series(p, eps):
    rng = _rng(10 + p)
    mask = np.add.outer(np.add.outer(np.arange(p + 1), np.arange(p + 1)), np.arange(p + 1)) <= p
    for _ in range(2):
        d = rng.standard_normal(3)
        Sj, Tj = reg_kernel_jets(d, eps, p)
        a = oracle.taylor_stokeslet_reg(d, eps, p)
        t = oracle.taylor_stresslet_reg(d, eps, p)
        for i in range(3):
            for j in range(3):
                ref = Sj[i][j].c
                np.testing.assert_allclose(a[i, j][mask], ref[mask], rtol=1e-11, atol=1e-12 * np.abs(ref).max())
                for l in range(3):
                    ref = Tj[i][j][l].c
                    np.testing.assert_allclose(t[i, j, l][mask], ref[mask], rtol=1e-11,
                                               atol=1e-12 * np.abs(ref).max())


def test_regularized_far_field_converges_geometrically():
    rng = _rng(30)
    yc = np.array([0.1, -0.2, 0.3])
    v = rng.standard_normal((40, 3))
    y = yc + 0.1 * v / np.linalg.norm(v, axis=1, keepdims=True) * rng.uniform(0, 1, (40, 1)) ** (1 / 3)
    f, h = rng.uniform(-1, 1, (40, 3)), rng.uniform(-1, 1, (40, 3))
    nu = rng.standard_normal((40, 3))
    x = yc + np.array([0.6, 0.5, -0.3])
    for eps in (0.02, 0.2):
        exact = oracle.direct_reg(y, f, h, nu, eps, targets=x[None])[0]
        errs = []
        for p in range(0, 9):
            Mf, Mt = oracle.moments(y, f, h, nu, yc, p)
            errs.append(np.linalg.norm(oracle.far_reg(x - yc, eps, p, Mf, Mt) - exact) / np.linalg.norm(exact))
        errs = np.array(errs)
        assert errs[-1] < 1e-8, errs
        assert np.all(errs[1:] < errs[:-1] * 1.5), errs


def test_regularized_far_field_at_tiny_eps_is_the_paper_far_field():
    """eps -> 0: the explicit regularized expansion equals eqs. (4.4) + (4.9)."""
    rng = _rng(31)
    for p in (0, 3, 8):
        d = rng.standard_normal(3) * 2.0
        Mf = rng.standard_normal((3,) + (p + 1,) * 3)
        Mt = rng.standard_normal((3, 3) + (p + 1,) * 3)
        u0 = oracle.far_contracted(d, p, Mf, Mt)
        np.testing.assert_allclose(oracle.far_reg(d, 1e-9, p, Mf, Mt), u0, rtol=1e-10, atol=1e-12 * np.abs(u0).max())


def test_regularized_treecode_limits():
    x, f, h, nu = inputs.uniform_cube(1200, 5007)
    tree = oracle.Tree(x, 60, True)
    tree.set_moments(f, h, nu, 5)
    eps = 0.02
    np.testing.assert_allclose(tree.treecode_reg(x, 1e-9, eps), oracle.direct_reg(x, f, h, nu, eps),
                               rtol=1e-12, atol=1e-12 * 1e3)
    u0 = tree.treecode(x, 0.5, 5)
    assert oracle.rel_l2(tree.treecode_reg(x, 0.5, 1e-9), u0) < 1e-11
    # and the truncation error of the regularized treecode behaves like the paper's
    ud = oracle.direct_reg(x, f, h, nu, eps)
    e3 = oracle.rel_l2(tree.treecode_reg(x, 0.5, eps, 3), ud)
    e5 = oracle.rel_l2(tree.treecode_reg(x, 0.5, eps, 5), ud)
    assert e5 < 0.5 * e3 < 1e-2
