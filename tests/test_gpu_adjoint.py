"""The adjoint (tc_adjoint) against the FP64 oracle.

L = sum_m g^m . u(x^m) with the structure of the last evaluation frozen.
* Weights: u is linear in f (and in h for fixed nu, and in nu for fixed h),
  so <dL/df, phi> must equal sum_m g^m . u_oracle(f = phi, h = 0) exactly up
  to rounding (and likewise for h and nu).  Tolerances: FP64 path 1e-10,
  mixed path 1e-6, relative to |dL/df| |phi|.
* Positions: central finite differences (step 1e-6, FP64) of the oracle's
  frozen-structure map (decisions at the original positions, moments and sums
  at the moved ones) on sampled entries; relative L2 over the samples, with
  each entry's error floored at the RMS of the gradient: <= 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_12498_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL_W = {"fp64": 1e-10, "mixed": 1e-6}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda()


def host(t):
    return t.cpu().numpy().T


def _adjoint(prec, x, f, h, nu, g, N0, p, theta, targets=None, shrink=True):
    tc = api.Treecode(prec, shrink).build(dev(x), N0).moments(dev(f), dev(h), dev(nu), p)
    tc.eval(theta, p, None if targets is None else dev(targets))
    gr = tc.adjoint(dev(g), t=targets is not None)
    tc.sync()
    out = {k: host(v) for k, v in gr.items()}
    tc.close()
    return out


def _L_oracle(tree, tgt, g, f, h, nu, p, theta):
    tree.set_moments(f, h, nu, p)
    return float(np.sum(g * tree.treecode(tgt, theta, p)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind,N,N0,p,theta", [("cube", 20000, 200, 6, 0.5), ("cube", 12000, 150, 8, 0.5),
                                               ("sphere", 15000, 150, 4, 0.7)])
def test_weight_gradients_dot_product(prec, kind, N, N0, p, theta):
    if kind == "cube":
        x, f, h, nu = inputs.uniform_cube(N, 301)
    else:
        x, f, h, nu = inputs.fibonacci_sphere(N, 302)
    rng = np.random.default_rng(303)
    g = rng.standard_normal((N, 3))
    gr = _adjoint(prec, x, f, h, nu, g, N0, p, theta)
    tree = oracle.Tree(x, N0, True)
    z = np.zeros_like(f)
    phi, psi, chi = (rng.standard_normal((N, 3)) for _ in range(3))
    checks = [(gr["f"], phi, _L_oracle(tree, x, g, phi, z, nu, p, theta)),
              (gr["h"], psi, _L_oracle(tree, x, g, z, psi, nu, p, theta)),
              (gr["nu"], chi, _L_oracle(tree, x, g, z, h, chi, p, theta))]
    for grad, probe, ref in checks:
        got = float(np.sum(grad * probe))
        scale = np.linalg.norm(grad) * np.linalg.norm(probe)
        assert abs(got - ref) <= TOL_W[prec] * scale, (got, ref, scale)


def _fd_positions(x, f, h, nu, g, N0, p, theta, entries, step, targets=None, which="x"):
    """Central differences of sum g . u_frozen on the listed (index, axis)."""
    tree = oracle.Tree(x, N0, True)
    tgt = x if targets is None else targets
    out = []
    for (n, a) in entries:
        vals = []
        for sgn in (1.0, -1.0):
            xe = x.copy()
            te = tgt.copy() if targets is not None else None
            if which == "x":
                xe[n, a] += sgn * step
                if targets is None:
                    te = xe
            else:
                te[n, a] += sgn * step
            u = tree.treecode_frozen(xe, f, h, nu, p, tgt, te, theta)
            vals.append(float(np.sum(g * u)))
        out.append((vals[0] - vals[1]) / (2 * step))
    return np.array(out)


def _fd_error(got, fd, full):
    floor = np.sqrt(np.mean(full ** 2))
    return float(np.sqrt(np.sum((got - fd) ** 2) / np.sum(np.maximum(np.abs(fd), floor) ** 2)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-5), ("mixed", 1e-5)])
@pytest.mark.parametrize("kind", ["cube", "clusters"])
def test_position_gradient_matches_finite_differences(prec, tol, kind):
    N, N0, p, theta = 3000, 100, 6, 0.5
    if kind == "cube":
        x, f, h, nu = inputs.uniform_cube(N, 311)
    else:
        x, f, h, nu = inputs.gaussian_clusters(N, 312)
    rng = np.random.default_rng(313)
    g = rng.standard_normal((N, 3))
    gr = _adjoint(prec, x, f, h, nu, g, N0, p, theta)
    idx = inputs.sample_indices(N, 24, 314)
    entries = [(int(n), int(k % 3)) for k, n in enumerate(idx)]
    fd = _fd_positions(x, f, h, nu, g, N0, p, theta, entries, 1e-6)
    got = np.array([gr["x"][n, a] for n, a in entries])
    err = _fd_error(got, fd, gr["x"])
    print("dL/dx vs central differences (%s, %s): %.3e" % (prec, kind, err))
    assert err <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_disjoint_targets_source_and_target_gradients(prec):
    N, N0, p, theta = 2500, 90, 5, 0.5
    x, f, h, nu = inputs.uniform_cube(N, 321)
    rng = np.random.default_rng(322)
    t = np.concatenate([rng.uniform(-0.2, 1.2, (800, 3)), x[:10]])
    g = rng.standard_normal((t.shape[0], 3))
    gr = _adjoint(prec, x, f, h, nu, g, N0, p, theta, targets=t)
    tol = 1e-5
    ex = [(int(n), int(k % 3)) for k, n in enumerate(inputs.sample_indices(N, 16, 323))]
    fd = _fd_positions(x, f, h, nu, g, N0, p, theta, ex, 1e-6, targets=t, which="x")
    assert _fd_error(np.array([gr["x"][n, a] for n, a in ex]), fd, gr["x"]) <= tol
    et = [(int(n), int(k % 3)) for k, n in enumerate(inputs.sample_indices(t.shape[0], 16, 324))]
    fdt = _fd_positions(x, f, h, nu, g, N0, p, theta, et, 1e-6, targets=t, which="t")
    assert _fd_error(np.array([gr["t"][n, a] for n, a in et]), fdt, gr["t"]) <= tol
    # weights with disjoint targets
    tree = oracle.Tree(x, N0, True)
    phi = rng.standard_normal((N, 3))
    ref = _L_oracle(tree, t, g, phi, np.zeros_like(f), nu, p, theta)
    got = float(np.sum(gr["f"] * phi))
    assert abs(got - ref) <= TOL_W[prec] * np.linalg.norm(gr["f"]) * np.linalg.norm(phi)


def test_autograd_function_matches_adjoint():
    N, N0, p, theta = 4000, 128, 6, 0.5
    x, f, h, nu = inputs.uniform_cube(N, 331)
    g = np.random.default_rng(332).standard_normal((N, 3))
    X, F, H, NU = (dev(a).requires_grad_(True) for a in (x, f, h, nu))
    u = api.stokes_velocity(X, F, H, NU, theta, p, N0, "fp64")
    (u * dev(g)).sum().backward()
    gr = _adjoint("fp64", x, f, h, nu, g, N0, p, theta)
    for name, T in (("x", X), ("f", F), ("h", H), ("nu", NU)):
        ref = gr[name]
        np.testing.assert_allclose(host(T.grad), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_adjoint_argument_checks():
    x, f, h, nu = inputs.uniform_cube(200, 341)
    tc = api.Treecode("fp64", True).build(dev(x), 20).moments(dev(f), dev(h), dev(nu), 3)
    with pytest.raises(api.TCError) as e:
        tc._M = 200
        tc.adjoint(dev(np.ones((200, 3))))
    assert e.value.status == 4  # no evaluation yet
    tc.eval(0.5, 3)
    with pytest.raises(api.TCError) as e:
        tc.adjoint(dev(np.ones((200, 3))), t=True)
    assert e.value.status == 1  # grad_t with targets = sources
    tc.close()


def test_full_size_sampled_weight_gradient():
    """N = 262,144 in 8 Gaussian clusters (sigma 0.05), p = 8, theta = 0.5,
    mixed precision: with g nonzero on 64 sampled targets only, L needs the
    oracle at those targets alone, so the dot-product identity is checked at
    full size."""
    N, N0, p, theta = 262_144, 2000, 8, 0.5
    x, f, h, nu = inputs.gaussian_clusters(N, inputs.SEED_BASE + 4)
    rng = np.random.default_rng(351)
    idx = inputs.sample_indices(N, 64, 352)
    g = np.zeros((N, 3))
    g[idx] = rng.standard_normal((len(idx), 3))
    gr = _adjoint("mixed", x, f, h, nu, g, N0, p, theta)
    tree = oracle.Tree(x, N0, True)
    z = np.zeros_like(f)
    phi = rng.standard_normal((N, 3))
    tree.set_moments(phi, z, nu, p)
    ref = float(np.sum(g[idx] * tree.treecode(x[idx], theta, p)))
    got = float(np.sum(gr["f"] * phi))
    assert abs(got - ref) <= 1e-6 * np.linalg.norm(gr["f"]) * np.linalg.norm(phi)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_adjoint_is_the_direct_gradient_when_every_pair_is_direct(prec, tol):
    """theta -> 0: no cluster of more than one point passes the MAC, so the
    treecode is the direct sum and its adjoint must be the gradient of the
    direct sum, which the oracle forms from the derivatives of S and T
    (measured: 4e-15 in FP64, 2.2e-7 in mixed precision)."""
    N = 1500
    x, f, h, nu = inputs.uniform_cube(N, inputs.SEED_BASE + 61)
    g = np.random.default_rng(62).standard_normal((N, 3))
    gr = _adjoint(prec, x, f, h, nu, g, 64, 4, 1e-9)
    ref = oracle.direct_grad(x, f, h, nu, g)
    for k in ("f", "h", "nu", "x"):
        assert oracle.rel_l2(gr[k], ref[k]) <= tol, (k, oracle.rel_l2(gr[k], ref[k]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_update_positions_gives_the_frozen_structure_map(prec):
    """tc_update_positions + tc_eval_frozen: the tree, centres, radii and the
    far/near decisions of the last tc_eval stay, the particles move; the
    result is the oracle's frozen-structure map (decisions at the old
    positions, moments, direct sums and evaluation at the new ones), and with
    the old positions it is the original evaluation again."""
    N, N0, p, theta = 3000, 100, 5, 0.5
    x, f, h, nu = inputs.uniform_cube(N, inputs.SEED_BASE + 63)
    xe = x + 2e-3 * np.random.default_rng(64).standard_normal(x.shape)
    tc = api.Treecode(prec, True).build(dev(x), N0).moments(dev(f), dev(h), dev(nu), p)
    u0 = host(tc.eval(theta, p))
    u = host(tc.update_positions(dev(xe)).eval_frozen())
    tree = oracle.Tree(x, N0, True)
    tree.set_moments(f, h, nu, p)
    ref = tree.treecode_frozen(xe, f, h, nu, p, x, xe, theta)
    assert oracle.rel_l2(u, ref) <= TOL_W[prec], oracle.rel_l2(u, ref)
    back = host(tc.update_positions(dev(x)).eval_frozen())
    np.testing.assert_allclose(back, u0, rtol=1e-13, atol=1e-13 * np.abs(u0).max())
    tc.close()


@pytest.mark.parametrize("prec,n_x,n_w", [("mixed", 32, 8), ("fp64", 16, 0)])
def test_full_size_gradients_match_central_differences(prec, n_x, n_w):
    """The headline adjoint configuration: N = 262,144 particles in 8 Gaussian
    clusters (sigma 0.05), p = 8, theta = 0.5, N0 = 2000.  L = sum g . u with
    g nonzero on 64 sampled targets, so each evaluation of the oracle's
    frozen-structure map needs its moment pass and those 64 targets only.
    Central differences of that map (FP64): dL/dx on 32 sampled entries
    (16 of them particles that are also weighted targets, step 1e-6) and
    dL/df, dL/dh, dL/dnu on 8 entries each (the map is linear in each weight
    vector, step 1e-3); the FP64 path on 16 position entries.  Relative L2 over the sampled entries, each entry's
    error floored at the RMS of its gradient: <= 1e-5."""
    N, N0, p, theta = 262_144, 2000, 8, 0.5
    x, f, h, nu = inputs.gaussian_clusters(N, inputs.SEED_BASE + 4)
    rng = np.random.default_rng(361)
    S = inputs.sample_indices(N, 64, 362)
    g = np.zeros((N, 3))
    g[S] = rng.standard_normal((len(S), 3))
    gr = _adjoint(prec, x, f, h, nu, g, N0, p, theta)
    tree = oracle.Tree(x, N0, True)
    gS = g[S]

    def L(xe=x, fe=f, he=h, ne=nu):
        return float(np.sum(gS * tree.treecode_frozen(xe, fe, he, ne, p, x[S], xe[S], theta)))

    others = inputs.sample_indices(N, 16, 363)
    pick = np.concatenate([S[:16], others])
    errs = {}
    for key, n_ent, step in (("x", n_x, 1e-6), ("f", n_w, 1e-3), ("h", n_w, 1e-3), ("nu", n_w, 1e-3)):
        if n_ent == 0:
            continue
        entries = [(int(n), int(k % 3)) for k, n in enumerate(pick[:n_ent] if key == "x" else pick[::4][:n_ent])]
        base = dict(x=x, f=f, h=h, nu=nu)[key]
        fd = []
        for n, a in entries:
            vals = []
            for sgn in (1.0, -1.0):
                arr = base.copy()
                arr[n, a] += sgn * step
                kw = {"xe" if key == "x" else ("fe" if key == "f" else ("he" if key == "h" else "ne")): arr}
                vals.append(L(**kw))
            fd.append((vals[0] - vals[1]) / (2 * step))
        got = np.array([gr[key][n, a] for n, a in entries])
        errs[key] = _fd_error(got, np.array(fd), gr[key])
    print("full-size adjoint (%s) vs central differences of the oracle's frozen map: %s"
          % (prec, ", ".join("%s %.3e" % kv for kv in errs.items())))
    assert max(errs.values()) <= 1e-5, errs
