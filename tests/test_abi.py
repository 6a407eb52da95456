"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/bae.h declares, and refuses to run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bae.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bae_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2502_05507_gb300 import build
    return build.build()


def test_header_declares_the_api():
    names = _declared()
    for n in ("bae_ctx_create", "bae_problem_create", "bae_potential_apply", "bae_solve", "bae_solve_batched",
              "bae_lgf_table", "bae_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2502_05507_gb300 import bae
    assert sorted(bae.EXPORTED) == _declared()


def test_no_gpu_fails_loudly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2502_05507_gb300 import bae
    L = bae.lib()
    h = ctypes.c_void_p()
    rc = L.bae_ctx_create(0, None, ctypes.byref(h))
    assert rc != bae.OK
    assert L.bae_last_error()
    opts = bae.Options()
    L.bae_default_options(ctypes.byref(opts))
    assert opts.tol == 1e-10 and opts.restart == 200 and opts.precision == bae.FP64
