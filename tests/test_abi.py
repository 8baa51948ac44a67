"""The C ABI library loads, exports every entry point declared in
include/tc.h, and its host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1811_12498_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1811_12498_gb300.build import build
        build()
    return _lib.lib()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 14
    from paper_1811_12498_gb300._lib import SIGNATURES
    for n in names:
        assert hasattr(lib, n), n
        assert n in SIGNATURES, n


def test_host_argument_checks_without_gpu(lib):
    # each of these returns before touching the CUDA runtime
    assert lib.tc_create(None, None) == 1
    assert b"out is NULL" in lib.tc_last_error(None)
    from paper_1811_12498_gb300._lib import TCConfig
    h = ctypes.c_void_p()
    bad = TCConfig(7, 1, None, 0, 0)
    assert lib.tc_create(ctypes.byref(h), ctypes.byref(bad)) == 1
    assert b"precision" in lib.tc_last_error(None)
    bad = TCConfig(0, 2, None, 0, 0)
    assert lib.tc_create(ctypes.byref(h), ctypes.byref(bad)) == 1
    assert lib.tc_build(None, None, 10, 5) == 1
    assert lib.tc_moments(None, None, None, None, 4) == 1
    assert lib.tc_eval(None, None, 10, 0.5, 4, None) == 1
    assert lib.tc_direct(None, None, None, None, 10, None, 10, 0, None, None) == 1
    assert b"NULL" in lib.tc_last_error(None)
    assert lib.tc_destroy(None) == 0
    assert lib.tc_sync(None) == 1
    assert lib.tc_tune(None, None, None, None, None, 10, None, 1, None, 1, None, 1, None, 1, 1e-3, None, None,
                       None) == 1
    assert b"ctx is NULL" in lib.tc_last_error(None)
    assert lib.tc_update_positions(None, None) == 1
    assert lib.tc_velocity_host(None, None, None, None, None, 10, 2, 0.5, 4, None) == 1
    assert lib.tc_eval_frozen(None, None) == 1
    assert lib.tc_direct_reg(None, None, None, None, 10, None, 10, 0.1, 0, None, None) == 1
    one = ctypes.c_void_p(1)
    assert lib.tc_direct_reg(one, one, one, one, 10, None, 10, 0.0, 0, None, one) == 1
    assert b"eps" in lib.tc_last_error(None)
    bad = TCConfig(0, 1, None, 0, 0, -1.0)
    assert lib.tc_create(ctypes.byref(h), ctypes.byref(bad)) == 1
    assert b"reg_eps" in lib.tc_last_error(None)
    assert lib.tc_fma_peak(0, None, None) == 1
    out = ctypes.c_double()
    assert lib.tc_fma_peak(5, None, ctypes.byref(out)) == 1
    assert b"precision" in lib.tc_last_error(None)


def test_oracle_and_library_share_no_code():
    """The CUDA sources never include or mention the oracle, and the oracle
    never includes the CUDA headers."""
    csrc = os.path.join(ROOT, "paper_1811_12498_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
    otext = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "tc_internal" not in otext and "tc.h" not in otext
    for f in os.listdir(os.path.join(ROOT, "paper_1811_12498_gb300")):
        if f.endswith(".py"):
            text = open(os.path.join(ROOT, "paper_1811_12498_gb300", f)).read()
            assert "import oracle" not in text and "from oracle" not in text, f


def declared_parameter_counts():
    """{entry point: number of parameters} from the prototypes in include/tc.h."""
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#define[^\n]*", "", src)
    out = {}
    for m in re.finditer(r"\b(tc_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """The ctypes table marshals exactly as many arguments as each C
    prototype declares (a mismatch would pass garbage through the ABI)."""
    from paper_1811_12498_gb300._lib import SIGNATURES
    counts = declared_parameter_counts()
    assert set(counts) == set(SIGNATURES), set(counts) ^ set(SIGNATURES)
    for name, n in counts.items():
        assert len(SIGNATURES[name][1]) == n, (name, n, len(SIGNATURES[name][1]))


def test_no_fallback_without_the_library_or_a_gpu(monkeypatch, tmp_path):
    """The binding never computes on the host: a missing libtc.so raises, and
    host (CPU) tensors are refused before any call reaches the library."""
    import torch
    from paper_1811_12498_gb300 import _lib, api
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libtc.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()
    with pytest.raises(TypeError, match="CUDA tensor"):
        api._vec3(torch.zeros(3, 4, dtype=torch.float64), "x", 4)
    with pytest.raises(TypeError, match="host"):
        api._host3([[0.0] * 4] * 3, "x", 4)
