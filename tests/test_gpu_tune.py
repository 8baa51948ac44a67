"""tc_tune (the fastest (theta, p, N0) of a grid that reaches a target error
E, Section 6's closing remark on tuning) through the C ABI: every error it
reports equals the oracle's E for that candidate (FP64 treecode at the sampled
particles against the FP64 direct sum), and the candidate it picks is the
fastest of those within the target."""
import numpy as np
import pytest

import oracle
from paper_1811_12498_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETAS, ORDERS, LEAVES = [0.4, 0.7], [2, 5], [150, 600]


def _system(N, seed):
    x, f, h, nu = inputs.uniform_cube(N, seed)
    return (x, f, h, nu), [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]


def _oracle_E(x, f, h, nu, idx, theta, p, N0, ud):
    tree = oracle.Tree(x, N0, True)
    tree.set_moments(f, h, nu, p)
    return oracle.rel_l2(tree.treecode(x[idx], theta, p), ud)


def test_tune_errors_match_oracle_and_best_is_fastest_within_target():
    from paper_1811_12498_gb300 import api

    (x, f, h, nu), d = _system(20000, inputs.SEED_BASE + 31)
    idx = inputs.sample_indices(x.shape[0], 400, 77)
    target = 2e-4
    res = api.Treecode("fp64", True).tune(*d, THETAS, ORDERS, LEAVES, idx, target)
    table = res["table"]
    assert len(table) == len(THETAS) * len(ORDERS) * len(LEAVES)
    # candidate order: leaf size outermost, theta innermost
    assert [r[:3] for r in table] == [(t, p, n0) for n0 in LEAVES for p in ORDERS for t in THETAS]
    ud = oracle.direct(x, f, h, nu, targets=x[idx])
    for t, p, n0, sec, E in table:
        Eo = _oracle_E(x, f, h, nu, idx, t, p, n0, ud)
        assert abs(E - Eo) <= 1e-6 * Eo + 1e-10, (t, p, n0, E, Eo)
        assert sec > 0
    ok = [r for r in table if r[4] <= target]
    assert ok, "the grid should contain a candidate within the target"
    assert res["best"] == min(ok, key=lambda r: r[3])[:3]
    # a target nothing reaches
    res = api.Treecode("fp64", True).tune(*d, [0.7], [2], [600], idx, 1e-12)
    assert res["best"] is None and res["table"][0][4] > 1e-12


def test_tune_mixed_precision_errors_and_bad_arguments():
    from paper_1811_12498_gb300 import api

    (x, f, h, nu), d = _system(20000, inputs.SEED_BASE + 32)
    idx = inputs.sample_indices(x.shape[0], 300, 78)
    r64 = api.Treecode("fp64", True).tune(*d, [0.5], [4, 6], [300], idx, 1e-3)["table"]
    r32 = api.Treecode("mixed", True).tune(*d, [0.5], [4, 6], [300], idx, 1e-3)["table"]
    for a, b in zip(r64, r32):
        # the mixed result differs from FP64 by ~1e-7 of |u|, far below E
        assert abs(a[4] - b[4]) <= 2e-6, (a, b)
    tc = api.Treecode("mixed", True)
    for args in (([1.5], [4], [300], idx, 1e-3), ([0.5], [13], [300], idx, 1e-3), ([0.5], [4], [0], idx, 1e-3),
                 ([0.5], [4], [300], [x.shape[0]], 1e-3), ([0.5], [4], [300], idx, 0.0), ([], [4], [300], idx, 1e-3)):
        with pytest.raises(api.TCError):
            tc.tune(*d, *args)
