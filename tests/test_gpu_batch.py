"""Batched evaluation (tc_batch_*): one persistent far and one persistent
near kernel over all systems, replayed from a CUDA graph, must give exactly
the per-system tc_eval result (same arithmetic in the same order), and that
result must match the FP64 oracle per system."""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_12498_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _systems(sizes, seed):
    xs, fs, hs, ns = [], [], [], []
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            x, f, h, nu = inputs.uniform_cube(int(n), seed + k)
        else:
            x, f, h, nu = inputs.fibonacci_sphere(int(n), seed + k)
        xs.append(x)
        fs.append(f)
        hs.append(h)
        ns.append(nu)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return xs, fs, hs, ns, off


def _seg(parts):
    return torch.from_numpy(np.ascontiguousarray(np.concatenate(parts).T)).cuda()


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-6), ("fp64", 1e-10)])
def test_batch_matches_separate_calls_and_oracle(prec, tol):
    sizes = [3000, 800, 5000, 33, 2500, 1200, 4100]
    xs, fs, hs, ns, off = _systems(sizes, 700)
    N0, p, theta = 200, 6, 0.6
    b = api.Batch(prec, True).build(_seg(xs), off, N0).moments(_seg(fs), _seg(hs), _seg(ns), p)
    u1 = b.eval(theta, p)
    u2 = b.eval(theta, p, out=u1.clone())  # replayed graph, fresh output
    sep = b.eval_separate(theta, p)
    torch.cuda.synchronize()
    u1h, u2h = u1.cpu().numpy(), u2.cpu().numpy()
    np.testing.assert_array_equal(u1h, u2h)
    for s in range(len(sizes)):
        us = u1h[:, off[s]:off[s + 1]]
        np.testing.assert_array_equal(us, sep[s].cpu().numpy())
        tree = oracle.Tree(xs[s], N0, True)
        tree.set_moments(fs[s], hs[s], ns[s], p)
        ref = tree.treecode(xs[s], theta, p)
        assert oracle.rel_l2(us.T, ref) <= tol
    info = b.info()
    assert info["far_warps"] in (1, 2) and info["near_warps"] in (2, 4, 8)
    b.close()


def test_batch_fp64_recurrence_option_matches_separate_calls():
    sizes = [2100, 700, 3300]
    xs, fs, hs, ns, off = _systems(sizes, 740)
    b = api.Batch("mixed", True, rec64=True).build(_seg(xs), off, 150).moments(_seg(fs), _seg(hs), _seg(ns), 8)
    u = b.eval(0.5, 8).cpu().numpy()
    sep = b.eval_separate(0.5, 8)
    for s in range(len(sizes)):
        np.testing.assert_array_equal(u[:, off[s]:off[s + 1]], sep[s].cpu().numpy())
        tree = oracle.Tree(xs[s], 150, True)
        tree.set_moments(fs[s], hs[s], ns[s], 8)
        assert oracle.rel_l2(u[:, off[s]:off[s + 1]].T, tree.treecode(xs[s], 0.5, 8)) <= 1e-6
    b.close()


def test_batch_without_graph_or_tuning_gives_the_same_result():
    sizes = [1500, 2700, 900]
    xs, fs, hs, ns, off = _systems(sizes, 720)
    res = []
    for tune, graph in ((True, True), (False, False), (False, True)):
        b = api.Batch("mixed", True, autotune=tune, graph=graph)
        b.build(_seg(xs), off, 150).moments(_seg(fs), _seg(hs), _seg(ns), 5)
        res.append(b.eval(0.5, 5).cpu().numpy())
        b.close()
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], res[2])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_with_tiny_systems_and_changing_order(prec):
    # systems of 1, 2 and 40 particles among larger ones (one near entry, one
    # leaf), evaluated at one order, replayed, then at another order and with
    # new weights (the graph is captured again): every system equals its own
    # tc_eval bit for bit and the oracle within the tolerance
    sizes = [1, 2, 1700, 40, 2600]
    xs, fs, hs, ns, off = _systems(sizes, 760)
    b = api.Batch(prec, True).build(_seg(xs), off, 64)
    tol = 1e-6 if prec == "mixed" else 1e-10
    for p, scale in ((4, 1.0), (4, 1.0), (7, -0.5)):
        b.moments(_seg([scale * f for f in fs]), _seg(hs), _seg(ns), p)
        u = b.eval(0.5, p).cpu().numpy()
        sep = b.eval_separate(0.5, p)
        assert np.all(u[:, 0] == 0.0)  # a single particle has nothing to sum
        for s in range(len(sizes)):
            us = u[:, off[s]:off[s + 1]]
            np.testing.assert_array_equal(us, sep[s].cpu().numpy())
            if sizes[s] > 2:
                tree = oracle.Tree(xs[s], 64, True)
                tree.set_moments(scale * fs[s], hs[s], ns[s], p)
                assert oracle.rel_l2(us.T, tree.treecode(xs[s], 0.5, p)) <= tol
    b.close()


def test_batch_rejects_bad_offsets():
    x = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    b = api.Batch("mixed")
    with pytest.raises(api.TCError):
        b.build(x, [0, 5, 5, 10], 4)  # empty system
    b.close()


def test_full_size_64_systems_batched_equals_separate_and_oracle():
    """The 64-system workload at full size (sizes log-uniform in [1e4, 5e5];
    even systems uniform cubes, odd ones Fibonacci spheres; p = 6, theta = 0.6,
    N0 = 2000; persistent kernels replayed from a CUDA graph with autotuned
    shapes, as the benchmark times it): equal bit for bit to 64 separate
    calls, and equal to the oracle on sampled targets of four systems."""
    sizes = inputs.batch_sizes(64, inputs.SEED_BASE + 5)
    parts = []
    for k, n in enumerate(sizes):
        gen = inputs.uniform_cube if k % 2 == 0 else inputs.fibonacci_sphere
        parts.append(gen(int(n), inputs.SEED_BASE + 500 + k))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    seg = [_seg([pp[c] for pp in parts]) for c in range(4)]
    N0, p, theta = 2000, 6, 0.6
    b = api.Batch("mixed", True).build(seg[0], off, N0).moments(seg[1], seg[2], seg[3], p)
    u = b.eval(theta, p)
    u = b.eval(theta, p, out=u)  # the replayed graph
    sep = b.eval_separate(theta, p)
    torch.cuda.synchronize()
    uh = u.cpu().numpy()
    for s in range(len(sizes)):
        np.testing.assert_array_equal(uh[:, off[s]:off[s + 1]], sep[s].cpu().numpy())
    for s in (0, 1, int(np.argmax(sizes)), int(np.argmin(sizes))):
        x, f, h, nu = parts[s]
        idx = inputs.sample_indices(x.shape[0], 16, 300 + s)
        tree = oracle.Tree(x, N0, True)
        tree.set_moments(f, h, nu, p)
        ref = tree.treecode(x[idx], theta, p)
        assert oracle.rel_l2(uh[:, off[s]:off[s + 1]].T[idx], ref) <= 1e-6, s
    b.close()
