"""Regularized Stokeslet and stresslet on the GPU (tc_config.reg_eps,
tc_direct_reg) against the oracle's regularized direct sum and treecode, the
same way as the paper's kernels: FP64 path within 1e-10 of the oracle
treecode (1e-12 for the direct sum), mixed path within 1e-6; at tiny eps the
regularized treecode is the treecode of eqs. (1.2a,b)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_12498_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda()


def host(u):
    return u.cpu().numpy().T


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("N,eps", [(2, 0.1), (33, 0.01), (1500, 0.002), (1500, 0.2)])
def test_direct_reg_matches_oracle(prec, tol, N, eps):
    x, f, h, nu = inputs.uniform_cube(N, 900 + N)
    u = host(api.direct_reg(dev(x), dev(f), dev(h), dev(nu), eps, precision=prec))
    ref = oracle.direct_reg(x, f, h, nu, eps)
    assert oracle.rel_l2(u, ref) <= tol, oracle.rel_l2(u, ref)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_direct_reg_disjoint_targets(prec, tol):
    x, f, h, nu = inputs.uniform_cube(1800, 931)
    rng = np.random.default_rng(932)
    t = np.concatenate([rng.uniform(-0.3, 1.3, (500, 3)), x[:7]])
    u = host(api.direct_reg(dev(x), dev(f), dev(h), dev(nu), 0.01, targets=dev(t), precision=prec))
    assert oracle.rel_l2(u, oracle.direct_reg(x, f, h, nu, 0.01, targets=t)) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind,N,N0,p,theta,eps", [("cube", 12000, 150, 4, 0.5, 0.005),
                                                   ("cube", 12000, 150, 8, 0.5, 0.05),
                                                   ("clusters", 10000, 120, 6, 0.6, 0.002),
                                                   ("sphere", 9000, 100, 5, 0.5, 0.01)])
def test_regularized_treecode_matches_oracle(prec, kind, N, N0, p, theta, eps):
    gen = {"cube": inputs.uniform_cube, "clusters": inputs.gaussian_clusters, "sphere": inputs.fibonacci_sphere}[kind]
    x, f, h, nu = gen(N, 941)
    tc = api.Treecode(prec, True, reg_eps=eps).build(dev(x), N0).moments(dev(f), dev(h), dev(nu), p)
    u = host(tc.eval(theta, p))
    tc.close()
    tree = oracle.Tree(x, N0, True)
    tree.set_moments(f, h, nu, p)
    ref = tree.treecode_reg(x, theta, eps, p)
    err = oracle.rel_l2(u, ref)
    print("regularized %s N %d p %d theta %.1f eps %g %s vs oracle: %.3e" % (kind, N, p, theta, eps, prec, err))
    assert err <= TOL[prec], err
    # and it is an approximation of the regularized direct sum
    idx = inputs.sample_indices(N, 300, 942)
    E = oracle.rel_l2(u[idx], oracle.direct_reg(x, f, h, nu, eps, targets=x[idx]))
    assert E < 1e-2, E


@pytest.mark.parametrize("p,rec64", [(9, False), (11, False), (8, True), (10, True)])
def test_regularized_mixed_far_field_variants(p, rec64):
    """Mixed precision above the register-resident order (p = 9, 11: the
    FP32 far field with its coefficients in shared memory) and with the FP64
    far field kept by rec64 at p >= 8: the oracle's regularized treecode
    within 1e-6."""
    x, f, h, nu = inputs.gaussian_clusters(9000, 991)
    tc = api.Treecode("mixed", True, rec64=rec64, reg_eps=0.004).build(dev(x), 100).moments(dev(f), dev(h), dev(nu), p)
    u = host(tc.eval(0.5, p))
    tc.close()
    tree = oracle.Tree(x, 100, True)
    tree.set_moments(f, h, nu, p)
    ref = tree.treecode_reg(x, 0.5, 0.004, p)
    err = oracle.rel_l2(u, ref)
    print("regularized clusters p = %d rec64 %s, mixed vs oracle: %.3e" % (p, rec64, err))
    assert err <= TOL["mixed"], err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_regularized_treecode_disjoint_targets(prec):
    x, f, h, nu = inputs.uniform_cube(8000, 951)
    rng = np.random.default_rng(952)
    t = np.concatenate([rng.uniform(-0.2, 1.2, (900, 3)), x[:5]])
    tc = api.Treecode(prec, True, reg_eps=0.01).build(dev(x), 100).moments(dev(f), dev(h), dev(nu), 6)
    u = host(tc.eval(0.5, 6, dev(t)))
    tc.close()
    tree = oracle.Tree(x, 100, True)
    tree.set_moments(f, h, nu, 6)
    assert oracle.rel_l2(u, tree.treecode_reg(t, 0.5, 0.01, 6)) <= TOL[prec]


def test_tiny_eps_gives_the_treecode_of_eqs_1_2():
    x, f, h, nu = inputs.uniform_cube(10000, 961)
    d = [dev(a) for a in (x, f, h, nu)]
    ur = host(api.Treecode("fp64", True, reg_eps=1e-10).build(d[0], 150).moments(d[1], d[2], d[3], 6).eval(0.5))
    u0 = host(api.Treecode("fp64", True).build(d[0], 150).moments(d[1], d[2], d[3], 6).eval(0.5))
    assert oracle.rel_l2(ur, u0) <= 1e-11


def test_regularized_paths_that_are_not_offered_say_so():
    x, f, h, nu = inputs.uniform_cube(500, 971)
    d = [dev(a) for a in (x, f, h, nu)]
    tc = api.Treecode("mixed", True, reg_eps=0.01).build(d[0], 50).moments(d[1], d[2], d[3], 4)
    tc.eval(0.5, 4)
    with pytest.raises(api.TCError) as e:
        tc.adjoint(dev(np.ones((500, 3))))
    assert e.value.status == 1 and "regularized" in str(e.value)
    tc.close()
    with pytest.raises(api.TCError):
        api.Treecode("mixed", True, reg_eps=-1.0)
    with pytest.raises(api.TCError):
        api.direct_reg(*d, 0.0)


def test_full_size_regularized_on_sampled_targets():
    """N = 10^6 uniform cube, p = 8, theta = 0.5, N0 = 2000, eps = 1e-3
    (a tenth of the mean spacing), mixed precision: the GPU treecode equals
    the oracle's at 200 sampled targets within 1e-6."""
    N, N0, p, theta, eps = 1_000_000, 2000, 8, 0.5, 1e-3
    x, f, h, nu = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    tc = api.Treecode("mixed", True, reg_eps=eps).build(dev(x), N0).moments(dev(f), dev(h), dev(nu), p)
    u = host(tc.eval(theta, p))
    tc.close()
    idx = inputs.sample_indices(N, 200, 981)
    tree = oracle.Tree(x, N0, True)
    tree.set_moments(f, h, nu, p)
    ref = tree.treecode_reg(x[idx], theta, eps, p)
    err = oracle.rel_l2(u[idx], ref)
    print("regularized N = 10^6, p = 8, mixed vs oracle on 200 targets: %.3e" % err)
    assert err <= 1e-6, err
