"""Table 1 of the paper reproduced on the GPU: test case 1 (Stokeslets and
stresslets at the centroids of an icosahedral triangulation of the unit
sphere, random weights in [-1, 1], shrunk clusters, N0 = 2000), with E taken
over ALL targets as in Section 6, against the FP64 direct sum on the GPU.
Column (a), N = 81920, in FP64 over the whole (theta, p) grid; column (b),
N = 327680, in mixed precision for theta = 0.5 and 0.8 (E >= 1e-6 there, well
above the mixed path's own 3e-7).  E is a statistic of random weights, so a
factor 1.5 is allowed (the oracle on 600 sampled targets lands within 0.87 to
1.18 of column (a))."""
import os

import numpy as np
import pytest

from paper_1811_12498_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_sphere_E.txt"), comments="#")
    return {(float(r[0]), int(r[1])): (float(r[2]), float(r[3])) for r in rows}


def _rel_l2(u, ref):
    return float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref))


@pytest.mark.parametrize("L, col, precision, thetas", [(6, 0, "fp64", (0.2, 0.5, 0.8)),
                                                        (7, 1, "mixed", (0.5, 0.8))])
def test_table1_error_on_gpu(L, col, precision, thetas):
    from paper_1811_12498_gb300 import api

    x, f, h, nu = inputs.icosahedral_sphere(L, inputs.SEED_BASE + 101)
    assert x.shape[0] == 20 * 4 ** L
    d = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]
    ud = api.direct(*d, precision="fp64")
    tc = api.Treecode(precision, True)
    tc.build(d[0], 2000).moments(d[1], d[2], d[3], 10)
    paper = _paper()
    for theta in thetas:
        for p in range(0, 11, 2):
            E = _rel_l2(tc.eval(theta, p), ud)
            e = paper[(theta, p)][col]
            assert e / 1.5 < E < e * 1.5, (L, theta, p, E, e)
