"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point declared in include/hisq.h, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hisq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hisq_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_00152_gb300 import build, hisq

    build.build()
    return hisq.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hisq_create", "hisq_load_links", "hisq_set_mass", "hisq_eigensolve", "hisq_solve",
                 "hisq_solve_device", "hisq_apply_dslash", "hisq_save_eigvecs", "hisq_load_eigvecs",
                 "hisq_last_error", "hisq_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2502_00152_gb300 import hisq

    protos = {p[0] for p in hisq._PROTOS}
    assert set(_declared()) == protos
    for n in _declared():
        assert hasattr(hisq, n), n


def test_library_is_built_for_sm_103a(lib):
    from paper_2502_00152_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVFLAGS)


def test_status_strings_and_defaults(lib):
    from paper_2502_00152_gb300 import hisq

    assert lib.hisq_status_string(0) == b"ok"
    assert lib.hisq_status_string(4) == b"not converged"
    p = hisq.hisq_default_solve_params()
    assert p.tol == 1e-10 and p.delta_rd == 0.1 and p.delta_tr == 1e-3  # Section 3 defaults
    assert p.precision_reliable == 64  # FP64 reliable updates (Section 3)
    e = hisq.hisq_default_eig_params()
    assert e.n_ev > 0 and e.n_kr > e.n_ev


@pytest.mark.parametrize("dims", [(4, 4, 4, 3), (2, 4, 4, 4), (4, 4, 4, 0), (6, 6, 5, 6)])
def test_create_rejects_bad_lattice(lib, dims):
    d = (ctypes.c_int * 4)(*dims)
    h = ctypes.c_void_p()
    assert lib.hisq_create(d, 1, 0, None, ctypes.byref(h)) == 1  # HISQ_ERR_INVALID_ARG
    assert not h.value


def test_null_context_is_rejected(lib):
    from paper_2502_00152_gb300 import hisq

    assert lib.hisq_set_mass(None, 0.1) == 1
    assert lib.hisq_solve(None, None, None, 1, None, None) == 1
    assert lib.hisq_eigensolve(None, None, None, None) == 1
    assert lib.hisq_last_error(None) == b"null context"


def test_missing_library_fails_loudly(tmp_path):
    from paper_2502_00152_gb300 import hisq

    with pytest.raises(RuntimeError, match="missing"):
        hisq.load_library(str(tmp_path / "libhisq.so"))
