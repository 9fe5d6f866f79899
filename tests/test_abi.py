"""The C-ABI library builds, loads and exports every symbol include/rqrcp.h declares.

No compute call is made (no GPU needed); argument validation paths that return
before touching the device are exercised where they need no handle.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|long long|size_t|void)\s+(rq_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2008_04447_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("rq_create", "rq_destroy", "rq_workspace_size", "rq_rqrcp", "rq_qr", "rq_trqrcp", "rq_tuxv"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in sorted(_declared()):
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2008_04447_gb300 import _lib
    assert set(_lib.exported_symbols()) == _declared()


def test_null_handle_is_rejected(lib):
    from paper_2008_04447_gb300 import _lib
    L = _lib.load()
    assert L.rq_destroy(None) == _lib.RQ_EHANDLE
    assert L.rq_rqrcp(None, 0, 1, 1, None, 1, 1, 0, 1, None, 1, None, None, None, None) == _lib.RQ_EHANDLE
    assert L.rq_launch_count(None) == -1
    assert L.rq_gemm_bf16(None, 4, 4, 4, None, 4, None, 4, None, 4, None, None) == _lib.RQ_EHANDLE


def test_header_constants_match_the_binding():
    from paper_2008_04447_gb300 import _lib
    txt = open(os.path.join(ROOT, "include", "rqrcp.h")).read()
    defs = dict(re.findall(r"^#define (RQ_\w+)\s+\(?(-?\d+)", txt, flags=re.M))
    for name in ("RQ_OK", "RQ_ENOMEM", "RQ_ECUDA", "RQ_ETIMEOUT", "RQ_ENOTIMPL", "RQ_EHANDLE", "RQ_ETOOBIG",
                 "RQ_FP64", "RQ_FP32", "RQ_MIXED", "RQ_MAX_B", "RQ_MAX_L"):
        assert int(defs[name]) == getattr(_lib, name), name


def test_block_and_sample_limits_are_argument_errors(lib):
    from paper_2008_04447_gb300 import _lib
    L = _lib.load()
    x = 1   # never dereferenced: the argument checks return first
    assert L.rq_rqrcp_noalloc(0, 300, 300, x, 300, _lib.RQ_MAX_B + 1, 8, 10, x, 300, x, x, x, None) == -6
    assert L.rq_rqrcp_noalloc(0, 300, 300, x, 300, _lib.RQ_MAX_B, _lib.RQ_MAX_L - _lib.RQ_MAX_B + 1, 10, x, 400,
                              x, x, x, None) == -7


def test_header_is_plain_c(lib, tmp_path):
    """include/rqrcp.h compiles as C99 (pedantic, warnings as errors), a C
    program links against the library, and its GPU-free calls agree with the
    Python binding's."""
    import subprocess
    from paper_2008_04447_gb300 import _lib
    src = os.path.join(ROOT, "tests", "native", "abi_c_check.c")
    libdir = os.path.join(ROOT, "paper_2008_04447_gb300")
    exe = str(tmp_path / "abi_c_check")
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    src, "-o", exe, "-L", libdir, "-lrqrcp", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = {r.split()[0]: r.split()[1:] for r in out if r.strip()}
    assert rows["entry_points"] == [str(len(_declared())), "missing", "0"]
    rc, prob = rows["latent_cdf"]
    assert rc == "0" and abs(float(prob) - _lib.rq_latent_cdf(4, 0.125)) < 1e-6
    assert rows["padding"] == ["0", str(_lib.rq_padding(0.125, 0.01))]
    assert rows["tiles_search"] == ["0", "64", "16", "1.000", "16"]
    assert rows["destroy_null"] == [str(_lib.RQ_EHANDLE)]


def test_gemm_bf16_rejects_an_output_overlapping_its_inputs(lib):
    """The overlap check runs on the host before any CUDA call, so it needs a
    handle only for its validity check: with NULL it is RQ_EHANDLE, and the
    overlap rule is exercised on a GPU in tests/test_gpu_gemm_bf16.py."""
    from paper_2008_04447_gb300 import _lib
    L = _lib.load()
    assert L.rq_gemm_bf16(None, 4, 4, 4, 4096, 4, 8192, 4, 4096, 4, None, None) == _lib.RQ_EHANDLE
