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


def test_batch_rejects_bad_offsets():
    x = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    b = api.Batch("mixed")
    with pytest.raises(api.TCError):
        b.build(x, [0, 5, 5, 10], 4)  # empty system
    b.close()
