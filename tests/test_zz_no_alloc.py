"""tc_direct_noalloc, the direct sum whose scratch lives in a fixed device
array instead of memory the call allocates (for callers that may not
allocate device memory on their own).  Called through the C ABI and checked
against the allocating tc_direct on the same inputs, twice in a row because
the calls share (and leave behind) the same scratch array.  Kept in a file
that pytest collects last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1811_12498_gb300 import api, inputs
from paper_1811_12498_gb300._lib import lib

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def _noalloc(x, f, h, nu, t, prec, u):
    N = x.shape[1]
    M = N if t is None else t.shape[1]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib().tc_direct_noalloc(_p(x), _p(f), _p(h), _p(nu), N, _p(t), M, prec, stream, _p(u))


@pytest.mark.parametrize("prec,tol", [(api.TC_FP64, 1e-12), (api.TC_MIXED, 1e-6)])
@pytest.mark.parametrize("N,M", [(20000, 3000), (300000, 40000), (777, None), (1_030_000, 10000)])
def test_noalloc_matches_allocating_direct_sum(prec, tol, N, M):
    x, f, h, nu = inputs.uniform_cube(N, 808 + N)
    dx, df, dh, dnu = (_dev(a) for a in (x, f, h, nu))
    t = None
    if M is not None:
        rng = np.random.default_rng(9)
        pts = np.concatenate([rng.uniform(-0.2, 1.2, (M - 5, 3)), x[:5]])  # includes coincident points
        t = _dev(pts)
    ref = api.direct(dx, df, dh, dnu, targets=t, precision=prec)
    torch.cuda.synchronize()
    Mt = N if M is None else M
    for _ in range(2):
        u = torch.full((3, Mt), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(dx, df, dh, dnu, t, prec, u)
        assert st == 0, lib().tc_last_error(None)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref))
        assert err <= tol, err


def test_noalloc_rejects_sizes_beyond_its_array():
    # 3M targets need 72 MB of partial sums, more than the 64 MiB array; the
    # buffers are real and full size, so nothing could be read out of bounds
    M = 3_000_000
    x, f, h, nu = inputs.uniform_cube(64, 5)
    dx, df, dh, dnu = (_dev(a) for a in (x, f, h, nu))
    t = torch.zeros((3, M), dtype=torch.float64, device="cuda")
    u = torch.zeros((3, M), dtype=torch.float64, device="cuda")
    st = _noalloc(dx, df, dh, dnu, t, api.TC_FP64, u)
    assert st == 1
    assert b"fixed array" in lib().tc_last_error(None)
