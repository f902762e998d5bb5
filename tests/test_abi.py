"""The C ABI library loads and exports every entry point include/*.h declares, and
host-side argument validation rejects bad problems before touching the GPU."""
import ctypes
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|void|long long|const char\s*\*)\s*\**\s*(dd_tv_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1901_00682_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("dd_tv_create", "dd_tv_solve", "dd_tv_energy", "dd_tv_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1901_00682_gb300 import _lib
    names = _declared_functions()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers exactly the declared surface
    assert names == set(_lib.SIGNATURES)


def test_params_struct_size_matches(lib):
    from paper_1901_00682_gb300 import _lib
    p = _lib.default_params()
    assert p.tau == 50.0 and abs(p.sigma - 0.01) < 1e-15 and p.tau0 == 10.0
    assert abs(p.sigma0 - 1 / 80) < 1e-15 and abs(p.gamma - 1 / 400) < 1e-15 and p.inner_iters == 10


@pytest.mark.parametrize("field,value,needle", [
    ("height", 0, "height"),
    ("sub_rows", 3, "sub_rows"),
    ("alpha", -1.0, "alpha"),
    ("alpha", math.nan, "alpha"),
    ("inner_iters", 0, "inner_iters"),
    ("inner_iters", 5000, "inner_iters"),
    ("sigma", 0.02, "tau * sigma"),
    ("sigma0", 0.1, "tau0 * sigma0"),
    ("gamma", 1.0, "gamma"),
    ("fidelity", 7, "fidelity"),
    ("path", 9, "path"),
])
def test_create_rejects_invalid(lib, field, value, needle):
    from paper_1901_00682_gb300 import _lib
    p = _lib.make_params(2, 2, 1, 1)
    setattr(p, field, value)
    h = ctypes.c_void_p()
    rc = lib.dd_tv_create(ctypes.byref(h), ctypes.byref(p))
    assert rc == _lib.EINVAL
    assert not h.value
    assert needle in lib.dd_tv_last_error(None).decode()


def test_create_rejects_tolerance_without_reference(lib):
    from paper_1901_00682_gb300 import _lib
    p = _lib.make_params(8, 8, 2, 2, outer_tol=1e-4)
    h = ctypes.c_void_p()
    assert lib.dd_tv_create(ctypes.byref(h), ctypes.byref(p)) == _lib.EINVAL
    assert "energy_ref" in lib.dd_tv_last_error(None).decode()


def test_null_handle_calls_are_safe(lib):
    from paper_1901_00682_gb300 import _lib
    assert lib.dd_tv_destroy(None) == _lib.OK
    assert lib.dd_tv_iterate(None, 1) == _lib.EINVAL
    assert lib.dd_tv_outer_count(None) == -1
    assert lib.dd_tv_fault_probe(None, 0, None) == _lib.EINVAL


def test_create_rejects_edge_counts_beyond_32_bit_numbering(lib):
    """The interface kernels number the edges in 32-bit integers: (N_r - 1) W + (N_c - 1) H
    must stay below 2^30 (here exactly 2^30), refused before any device call."""
    from paper_1901_00682_gb300 import _lib
    p = _lib.make_params(32768, 32768, 16385, 16385)
    h = ctypes.c_void_p()
    rc = lib.dd_tv_create(ctypes.byref(h), ctypes.byref(p))
    assert rc == _lib.EINVAL and not h.value
    assert "interface edges" in lib.dd_tv_last_error(None).decode()


def _batch_args(**over):
    from paper_1901_00682_gb300 import _lib
    im = dict(height=256, width=128, fidelity=_lib.L2, alpha=10.0, c1=0.0, c2=0.0, tau=0.0, sigma=0.0)
    pa = dict(tile=128, inner_iters=10, tau0=10.0, sigma0=1 / 80, variant=0)
    for k, v in over.items():
        (im if k in im else pa)[k] = v
    arr = (_lib.BatchImage * 2)()
    arr[0] = _lib.BatchImage(**im)
    arr[1] = _lib.BatchImage(128, 128, _lib.SEG, 20.0, 0.2, 0.8, 1.0, 0.5)
    return arr, _lib.BatchParams(**pa)


@pytest.mark.parametrize("field,value,code,needle", [
    ("height", 200, "EINVAL", "multiples of the subdomain side 128"),
    ("width", 0, "EINVAL", "multiples of the subdomain side 128"),
    ("fidelity", 9, "EINVAL", "fidelity"),
    ("alpha", -2.0, "EINVAL", "alpha"),
    ("alpha", math.inf, "EINVAL", "alpha"),
    ("tau", 10.0, "EINVAL", "tau sigma"),          # tau given, sigma 0
    ("tile", 96, "EUNSUPPORTED", "64 or 128"),
    ("inner_iters", 0, "EINVAL", "inner_iters"),
    ("sigma0", 0.1, "EINVAL", "tau0 sigma0"),
    ("variant", 1, "EINVAL", "variant"),
])
def test_batch_create_rejects_invalid(lib, field, value, code, needle):
    """The batched solver validates every image and the shared parameters on the host
    and refuses bad ones before any device call."""
    from paper_1901_00682_gb300 import _lib
    arr, bp = _batch_args(**{field: value})
    h = ctypes.c_void_p()
    rc = lib.dd_tv_batch_create(ctypes.byref(h), arr, 2, ctypes.byref(bp))
    assert rc == getattr(_lib, code) and not h.value
    assert needle in lib.dd_tv_batch_last_error(None).decode()


def test_batch_variant_2_needs_tile_128(lib):
    from paper_1901_00682_gb300 import _lib
    arr, bp = _batch_args(tile=64, height=128, variant=2)
    h = ctypes.c_void_p()
    assert lib.dd_tv_batch_create(ctypes.byref(h), arr, 2, ctypes.byref(bp)) == _lib.EINVAL and not h.value
    assert "variant" in lib.dd_tv_batch_last_error(None).decode()


def test_batch_create_rejects_empty_batch(lib):
    from paper_1901_00682_gb300 import _lib
    arr, bp = _batch_args()
    h = ctypes.c_void_p()
    assert lib.dd_tv_batch_create(ctypes.byref(h), arr, 0, ctypes.byref(bp)) == _lib.EINVAL and not h.value
    assert lib.dd_tv_batch_destroy(None) == _lib.OK
    assert lib.dd_tv_batch_iterate(None, 1) == _lib.EINVAL


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: loading a missing library raises ImportError."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1901_00682_gb300 import _lib\n"
            "try:\n    _lib.load(%r)\nexcept ImportError as e:\n    print('ImportError', e)\n") % (
        ROOT, str(tmp_path / "libddtv.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ImportError"), r.stdout + r.stderr


def test_product_code_never_touches_the_oracle():
    """The library and its binding share nothing with the oracle: no module of the
    package imports it, and no CUDA source includes or names its files."""
    pkg = os.path.join(ROOT, "paper_1901_00682_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")):
        src = open(path).read()
        assert not re.search(r"^\s*(import oracle|from oracle)", src, flags=re.M), path
    for path in glob.glob(os.path.join(pkg, "csrc", "*")):
        src = open(path).read()
        assert "dd_tv_oracle" not in src and "oracle/" not in src, path


@pytest.mark.parametrize("rows,begin,end,path,code,needle", [
    (512, 2, 2, "fused", "EINVAL", "nonempty range"),
    (512, 0, 5, "fused", "EINVAL", "nonempty range"),
    (512, -1, 2, "fused", "EINVAL", "start at 0"),
    (502, 0, 2, "fused", "EINVAL", "equal height"),
    (512, 0, 2, "plain", "EUNSUPPORTED", "fused path"),
])
def test_create_shard_rejects_invalid(lib, rows, begin, end, path, code, needle):
    """A row-block shard is validated on the host before any device call."""
    from paper_1901_00682_gb300 import _lib
    p = _lib.make_params(rows, 256, 4, 2, path=path)
    h = ctypes.c_void_p()
    assert lib.dd_tv_create_shard(ctypes.byref(h), ctypes.byref(p), begin, end) == getattr(_lib, code)
    assert not h.value
    assert needle in lib.dd_tv_last_error(None).decode()
