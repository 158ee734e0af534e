"""The C-ABI library builds, loads without a GPU, and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cggm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cggm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1509_04681_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cggm_solve", "cggm_objective", "cggm_grad", "cggm_create", "cggm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    import paper_1509_04681_gb300 as cg
    assert set(cg.EXPORTED) == set(declared_functions())


def test_status_strings_and_defaults(lib):
    import paper_1509_04681_gb300 as cg
    o = cg.opts_default()
    assert o.tol == 0.01 and o.max_iter == 1000 and o.penalize_diag == 1
    assert o.ls_sigma == 1e-3 and o.ls_beta == 0.5 and o.ls_max_trials == 50
    lib.cggm_status_string.restype = ctypes.c_char_p
    assert lib.cggm_status_string(-2) == b"matrix not positive definite"


def test_bad_device_is_einval_not_a_crash(lib):
    h = ctypes.c_void_p()
    assert lib.cggm_create(ctypes.byref(h), 12345, None) == -1


def test_sm103a_only_sources():
    """The build names one architecture, sm_103a, and the CUDA sources hold no
    compatibility paths (Triton, other architectures)."""
    from paper_1509_04681_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for src in build.sources():
        s = open(src).read()
        assert "triton" not in s.lower()
        assert "__CUDA_ARCH__ <" not in s


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the compiled library every entry point raises: there is no fallback."""
    import paper_1509_04681_gb300.cggm as m
    monkeypatch.setattr(m, "_LIB", None)
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "libcggm.so"))
    with pytest.raises(ImportError):
        m.opts_default()
    with pytest.raises(ImportError):
        m.Context(0)
    with pytest.raises(ImportError):
        m.partition_columns(3, [0], [1], 2)


def test_no_cpu_fallback_in_the_package():
    """The package never imports the oracle or computes on the host in place of the
    library: its modules name neither the oracle nor numpy linear algebra."""
    import paper_1509_04681_gb300 as pkg
    pkg_dir = os.path.dirname(pkg.__file__)
    for f in os.listdir(pkg_dir):
        if f.endswith(".py"):
            src = open(os.path.join(pkg_dir, f)).read()
            assert "oracle" not in src, f
            assert "np.linalg" not in src and "scipy" not in src, f


def test_free_coo_accepts_null_and_empty_lists(lib):
    """cggm_free_coo is host code: NULL and an empty list are ignored, no GPU needed."""
    import paper_1509_04681_gb300 as cg
    lib.cggm_free_coo.argtypes = [ctypes.POINTER(cg.cggm_coo)]
    lib.cggm_free_coo.restype = None
    lib.cggm_free_coo(None)
    e = cg.cggm_coo()
    lib.cggm_free_coo(ctypes.byref(e))
    assert e.nnz == 0 and not e.row and not e.col and not e.val


def test_binding_lists_the_nonzeros_of_dense_warm_starts():
    """The binding's marshalling of a dense warm start into a coordinate list: Lambda by
    its upper triangle, Theta in full, row-major, zeros left out; and back."""
    import numpy as np
    import paper_1509_04681_gb300.cggm as m
    L = np.array([[2.0, 0.5, 0.0], [0.5, 3.0, -1.0], [0.0, -1.0, 4.0]])
    c = m._CooIn(L, upper=True)
    assert c.coo.nnz == 5
    assert list(zip(c.r, c.c, c.v)) == [(0, 0, 2.0), (0, 1, 0.5), (1, 1, 3.0), (1, 2, -1.0),
                                        (2, 2, 4.0)]
    np.testing.assert_array_equal(m.coo_to_dense((c.r, c.c, c.v), (3, 3), symmetric=True), L)
    T = np.array([[0.0, 1.5], [-2.0, 0.0]])
    t = m._CooIn(T, upper=False)
    assert list(zip(t.r, t.c, t.v)) == [(0, 1, 1.5), (1, 0, -2.0)]
    np.testing.assert_array_equal(m.coo_to_dense((t.r, t.c, t.v), (2, 2)), T)
    trip = m._CooIn((np.array([1]), np.array([0]), np.array([7.0])), upper=False)
    assert trip.coo.nnz == 1 and trip.v[0] == 7.0
