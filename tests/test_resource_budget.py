"""Register budget that lets the FP64 leaf moment pass run beside the near
field.  In mixed precision the near field (k_near_leaf<NearOpU>) keeps all
but kLeafFreeBlocks of the blocks that fit on an SM resident, and the leaf
pass (k_moments<1>, one block per SM at p <= 8) must fit in the registers
those blocks leave; otherwise it waits for the near field to end and the
moments are no longer hidden.  The register counts come from ptxas's
resource report (-Xptxas -v) of the sm_103a build; no GPU is needed."""
import math
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_12498_gb300", "csrc")
REGS_PER_SM = 65536
ALLOC_UNIT = 256  # registers are allocated per warp in units of 256


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def _registers(src, tmp_path):
    """{mangled kernel name: registers per thread} from ptxas -v."""
    cmd = [_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I",
           os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o",
           str(tmp_path / (src + ".o"))]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    regs, name = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            regs[name] = int(m.group(1))
            name = None
    return regs


def _constant(src, name):
    text = open(os.path.join(CSRC, src)).read()
    return int(re.search(r"constexpr int %s = (\d+);" % name, text).group(1))


def _warp_regs(r):
    return math.ceil(r * 32 / ALLOC_UNIT) * ALLOC_UNIT


@pytest.mark.skipif(_nvcc() is None, reason="nvcc not found")
def test_leaf_moment_pass_fits_beside_the_near_field(tmp_path):
    near = [v for k, v in _registers("tc_near.cu", tmp_path).items() if "k_near_leaf" in k and "NearOpU" in k]
    mom = [v for k, v in _registers("tc_moments.cu", tmp_path).items() if "k_momentsILi1E" in k]
    assert len(near) == 1 and len(mom) == 1, (near, mom)
    near_warps = _constant("tc_nearpair.cuh", "kLeafWarps")
    free = _constant("tc_nearpair.cuh", "kLeafFreeBlocks")
    mom_threads = _constant("tc_moments.cu", "kLeafMomThreads")
    near_block = near_warps * _warp_regs(near[0])
    mom_block = (mom_threads // 32) * _warp_regs(mom[0])
    fit = REGS_PER_SM // near_block
    resident = max(fit - free, 1) * near_block
    assert resident + mom_block <= REGS_PER_SM, (
        "near field %d registers x %d resident blocks + leaf pass %d registers x %d threads exceed the SM" %
        (near[0], max(fit - free, 1), mom[0], mom_threads))
    # one coefficient per thread (S = 1) up to p = 8: C(p+3, 3) = 165
    assert mom_threads >= math.comb(8 + 3, 3)
