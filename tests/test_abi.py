"""CPU checks of the C ABI: the library builds, loads and exports what the header declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(fdas_[a-z0-9_]+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1805_12280_gb300 as fd
    return fd.load()


def test_header_declares_entry_points():
    names = _declared_symbols()
    for must in ("fdas_plan_create", "fdas_convolve", "fdas_destroy", "fdas_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1805_12280_gb300 as fd
    out = subprocess.run(["nm", "-D", "--defined-only", fd.fdas.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s+(fdas_\w+)", out))
    declared = _declared_symbols()
    assert declared <= exported, f"declared but not exported: {declared - exported}"
    for name in declared:
        assert hasattr(lib, name)
    # the binding declares a signature for each header entry point
    assert declared <= set(fd.fdas.SIGNATURES)


def test_strerror_and_version_without_gpu(lib):
    import paper_1805_12280_gb300 as fd
    assert fd.fdas_version().startswith("fdas-gb300")
    assert lib.fdas_strerror(0) == b"ok"
    assert lib.fdas_strerror(-1) == b"invalid argument"
    assert lib.fdas_strerror(-4) == b"timed out"


def test_argument_errors_without_gpu(lib):
    import ctypes
    import paper_1805_12280_gb300 as fd
    # null handles and out-of-range sizes are rejected before any CUDA call
    assert lib.fdas_convolve(None, None, 10, None, None) == fd.fdas.FDAS_ERR_INVALID_ARG
    assert lib.fdas_destroy(None) == fd.fdas.FDAS_ERR_INVALID_ARG
    assert lib.fdas_plan_tpl_per_cta(None, 10) == fd.fdas.FDAS_ERR_INVALID_ARG
    assert lib.fdas_selftest_wait_timeout(None, 1.0, None) == fd.fdas.FDAS_ERR_INVALID_ARG
    assert lib.fdas_fdfir_convolve(None, None, 10, None, None) == fd.fdas.FDAS_ERR_INVALID_ARG
    assert lib.fdas_fdfir_destroy(None) == fd.fdas.FDAS_ERR_INVALID_ARG
    ff = ctypes.c_void_p()
    assert lib.fdas_fdfir_create(ctypes.byref(ff), (1 << 23) - 419, ctypes.c_void_p(1), 85, 421) == \
        fd.fdas.FDAS_ERR_INVALID_ARG                    # n_max + K - 1 > 2^23
    assert lib.fdas_fdfir_create(ctypes.byref(ff), 100, None, 85, 421) == fd.fdas.FDAS_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    opts = fd.fdas.fdas_opts(3000, 0, 0, 0)
    assert lib.fdas_plan_create(ctypes.byref(h), 100, ctypes.c_void_p(1), 85, 421, ctypes.byref(opts)) == \
        fd.fdas.FDAS_ERR_INVALID_ARG
    assert b"seg_len" in lib.fdas_last_error()
    opts = fd.fdas.fdas_opts(2048, 0, 0, 0)
    assert lib.fdas_plan_create(ctypes.byref(h), 100, ctypes.c_void_p(1), 85, 2045, ctypes.byref(opts)) == \
        fd.fdas.FDAS_ERR_INVALID_ARG
    assert lib.fdas_plan_create(ctypes.byref(h), 0, ctypes.c_void_p(1), 85, 421, None) == \
        fd.fdas.FDAS_ERR_INVALID_ARG
    opts = fd.fdas.fdas_opts(2048, 0, 7, 0)
    assert lib.fdas_plan_create(ctypes.byref(h), 100, ctypes.c_void_p(1), 85, 421, ctypes.byref(opts)) == \
        fd.fdas.FDAS_ERR_UNSUPPORTED
    # template groups: FP32 form only, no autotuning, flag 0 or 1
    for prec, tune, grp, code in ((1, 0, 1, fd.fdas.FDAS_ERR_UNSUPPORTED), (0, 1, 1, fd.fdas.FDAS_ERR_UNSUPPORTED),
                                  (0, 0, 2, fd.fdas.FDAS_ERR_INVALID_ARG)):
        opts = fd.fdas.fdas_opts(2048, 0, prec, tune, grp)
        assert lib.fdas_plan_create(ctypes.byref(h), 100, ctypes.c_void_p(1), 85, 421, ctypes.byref(opts)) == code


def test_product_package_never_imports_oracle():
    # the product path must not route through the CPU oracle
    pkg = os.path.join(ROOT, "paper_1805_12280_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src and "fdas_oracle" not in src, fn


def test_harmonic_sum_argument_errors_without_gpu(lib):
    import ctypes
    import paper_1805_12280_gb300 as fd
    bad = fd.fdas.FDAS_ERR_INVALID_ARG
    thr = (ctypes.c_float * 6)(7, 10, 16, 25, 40, 66)
    P, cnt, cand = ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(1024)   # never dereferenced
    ok = dict(plane=P, m=85, n=1000, bin0=210, H=8, thr=thr, cand=cand, max_cand=10, count=cnt)

    def call(**kw):
        a = {**ok, **kw}
        return lib.fdas_harmonic_sum(a["plane"], a["m"], a["n"], a["bin0"], a["H"], a["thr"], a["cand"],
                                     a["max_cand"], a["count"], None)
    for kw in (dict(plane=None), dict(count=None), dict(thr=None), dict(cand=None),
               dict(m=84), dict(m=0), dict(n=0), dict(bin0=1000), dict(bin0=-1),
               dict(H=3), dict(H=64), dict(H=0), dict(max_cand=-1),
               dict(plane=ctypes.c_void_p(258)), dict(count=ctypes.c_void_p(516))):
        assert call(**kw) == bad, kw
    assert b"power of two" in (call(H=3), lib.fdas_last_error())[1]


def test_harmonic_binding_checks_without_gpu():
    torch = pytest.importorskip("torch")
    import paper_1805_12280_gb300 as fd
    with pytest.raises(ValueError):
        fd.harmonic_sum(torch.zeros((85, 100), dtype=torch.float32), 10, 8)        # host tensor
    with pytest.raises(ValueError):
        fd.harmonic_sum(torch.zeros(100, dtype=torch.float32), 10, 8)              # not 2-D
    with pytest.raises(ValueError):
        fd.harmonic_sum(torch.zeros((85, 100), dtype=torch.float64), 10, 8)        # not float32
