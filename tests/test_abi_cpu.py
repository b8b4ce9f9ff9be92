"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/espnmf.h declares; argument validation
that needs no device; and no silent CPU path (without a GPU the calls that
need one fail with ESPNMF_ERR_CUDA)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_05237_gb300 import build
    build.build()
    import paper_1510_05237_gb300 as E
    return E.load()


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(espnmf_[A-Za-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_resolves_every_symbol(lib):
    import paper_1510_05237_gb300 as E
    assert all(E.exported_symbols().values())
    assert set(E.exported_symbols()) <= set(header_functions())


def test_status_strings(lib):
    lib.espnmf_status_string.restype = ctypes.c_char_p
    assert lib.espnmf_status_string(0) == b"ESPNMF_OK"
    assert lib.espnmf_status_string(3) == b"ESPNMF_ERR_SINGULAR"


def test_argument_validation_before_any_device_work(lib):
    import paper_1510_05237_gb300 as E
    from gen import small_zipf, uniform_init
    A = small_zipf(1)
    U0 = uniform_init(A.n, 4, 1)
    for kw, code in [(dict(k=0), E.ERR_INVALID_ARG), (dict(k=A.m + 1), E.ERR_INVALID_ARG),
                     (dict(t_u=-1), E.ERR_INVALID_ARG), (dict(mode=7), E.ERR_INVALID_ARG),
                     (dict(compute=E.BF16), E.ERR_UNSUPPORTED)]:
        args = dict(k=4, t_u=10, t_v=10, mode=E.TOPT_COLUMN, compute=E.F64)
        args.update(kw)
        with pytest.raises(E.EspnmfError) as ei:
            E.espnmf_init(A.rowptr, A.colidx, A.val, A.n, A.m, args["k"], args["t_u"],
                          args["t_v"], args["mode"], args["compute"], U0)
        assert ei.value.status == code


def test_no_cpu_fallback(lib):
    """With no CUDA device the library refuses to work instead of falling
    back to a host implementation."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1510_05237_gb300 as E
    from gen import small_zipf, uniform_init
    A = small_zipf(1)
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_init(A.rowptr, A.colidx, A.val, A.n, A.m, 4, 10, 10, E.TOPT_COLUMN, E.F64,
                      uniform_init(A.n, 4, 1))
    assert ei.value.status == E.ERR_CUDA


def test_library_is_built_for_sm103a():
    from paper_1510_05237_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_sequential_validates_and_needs_a_gpu(lib):
    """espnmf_sequential rejects bad arguments before any device work and,
    without a CUDA device, fails instead of running on the host."""
    import ctypes
    import numpy as np
    import paper_1510_05237_gb300 as E
    from paper_1510_05237_gb300 import binding as B
    from gen import small_zipf, uniform_init
    A = small_zipf(1)
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    csr = B._CSR(A.n, A.m, len(ci), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, E.F64, 0)
    u0 = np.ascontiguousarray(uniform_init(A.n, 1, 1)[:, 0])
    out_u = np.zeros(A.n * 4)
    out_v = np.zeros(A.m * 4)

    def call(k, iters, k2=1):
        return lib.espnmf_sequential(ctypes.byref(csr), k, k2, 10, 10, iters, E.F64,
                                     ctypes.c_void_p(u0.ctypes.data), E.F64, 0,
                                     ctypes.c_void_p(out_u.ctypes.data),
                                     ctypes.c_void_p(out_v.ctypes.data), None, None)
    assert call(0, 1) == E.ERR_INVALID_ARG
    assert call(2, 0) == E.ERR_INVALID_ARG
    assert call(A.m + 1, 1) == E.ERR_INVALID_ARG
    assert call(3, 1, k2=2) == E.ERR_INVALID_ARG      # k not a multiple of k2
    assert call(2, 1, k2=0) == E.ERR_INVALID_ARG
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert call(2, 1) == E.ERR_CUDA


def test_checked_flags_entry_point(lib):
    """espnmf_checked_flags: in the regular build it reports UNSUPPORTED and
    clears the output; in the checked build without a GPU it fails with
    ERR_CUDA instead of returning made-up flags."""
    import ctypes
    import os
    import subprocess
    import sys
    import paper_1510_05237_gb300 as E
    f = ctypes.c_uint32(7)
    assert lib.espnmf_checked_flags(ctypes.byref(f)) == E.ERR_UNSUPPORTED and f.value == 0
    assert lib.espnmf_checked_flags(None) == E.ERR_INVALID_ARG
    from paper_1510_05237_gb300 import build as B
    if not os.path.exists(B.LIB_CHECKED):
        pytest.skip("checked build not present")
    code = ("import ctypes, paper_1510_05237_gb300 as E\n"
            "from paper_1510_05237_gb300 import binding as b\n"
            "assert b.library_path().endswith('libespnmf_checked.so')\n"
            "f = ctypes.c_uint32(7)\n"
            "print(E.load().espnmf_checked_flags(ctypes.byref(f)))\n")
    env = dict(os.environ, ESPNMF_CHECKED="1", CUDA_VISIBLE_DEVICES="")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.strip().splitlines()[-1]) == E.ERR_CUDA
