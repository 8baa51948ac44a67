"""Failure paths and measurement helpers of the C ABI on the GPU.

* Out of memory is injected on the host (tc_fail_allocations): the call that
  needed the allocation returns TC_ENOMEM with a message, nothing runs on the
  device, and the same context works again once the injection is off.
* tc_fma_peak measures the FP32 and FP64 FMA rates the roofline fractions are
  taken against; they must lie near the part's unit counts x clock.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_12498_gb300 import api, inputs

pytestmark = pytest.mark.gpu

ENOMEM = 2


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda()


@pytest.fixture(autouse=True)
def _injection_off():
    api.fail_allocations(-1)
    yield
    api.fail_allocations(-1)


def test_out_of_memory_at_create_is_reported():
    api.fail_allocations(0)
    with pytest.raises(api.TCError) as e:
        api.Treecode("mixed")
    assert e.value.status == ENOMEM and "out of memory" in str(e.value)


@pytest.mark.parametrize("after", [0, 3, 9])
def test_out_of_memory_during_build_leaves_a_usable_context(after):
    N, N0, p, theta = 3000, 100, 5, 0.5
    x, f, h, nu = inputs.uniform_cube(N, 401)
    tc = api.Treecode("mixed")
    api.fail_allocations(after)
    with pytest.raises(api.TCError) as e:
        tc.build(dev(x), N0)
    assert e.value.status == ENOMEM
    with pytest.raises(api.TCError):  # nothing was built
        tc.moments(dev(f), dev(h), dev(nu), p)
    api.fail_allocations(-1)
    tc.build(dev(x), N0).moments(dev(f), dev(h), dev(nu), p)
    u = tc.eval(theta, p).cpu().numpy().T
    tree = oracle.Tree(x, N0, True)
    tree.set_moments(f, h, nu, p)
    assert oracle.rel_l2(u, tree.treecode(x, theta, p)) <= 1e-6
    tc.close()


def test_out_of_memory_in_direct_and_eval():
    N = 2000
    x, f, h, nu = inputs.uniform_cube(N, 402)
    api.fail_allocations(0)
    with pytest.raises(api.TCError) as e:
        api.direct(dev(x), dev(f), dev(h), dev(nu), precision="mixed")
    assert e.value.status == ENOMEM
    api.fail_allocations(-1)
    tc = api.Treecode("fp64")
    tc.build(dev(x), 64).moments(dev(f), dev(h), dev(nu), 4)
    api.fail_allocations(0)
    with pytest.raises(api.TCError) as e:
        tc.eval(0.5, 4)
    assert e.value.status == ENOMEM
    api.fail_allocations(-1)
    u = tc.eval(0.5, 4).cpu().numpy().T
    tree = oracle.Tree(x, 64, True)
    tree.set_moments(f, h, nu, 4)
    assert oracle.rel_l2(u, tree.treecode(x, 0.5, 4)) <= 1e-10
    tc.close()


def test_measured_fma_peaks_are_near_the_unit_counts():
    """FP32: 128 FMA lanes per SM, FP64: 2 per SM (GB300), at most 2.07 GHz."""
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    f32 = api.fma_peak("mixed")
    f64 = api.fma_peak("fp64")
    nominal32 = sms * 128 * 2 * 2.07e9 / 1e12
    print("measured FP32 %.1f TFLOP/s, FP64 %.3f TFLOP/s (nominal FP32 %.1f)" % (f32, f64, nominal32))
    assert 0.5 * nominal32 < f32 < 1.05 * nominal32
    assert 0.0 < f64 < f32
