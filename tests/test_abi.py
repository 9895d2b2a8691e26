"""The C ABI library builds, loads and exports every function that
include/bem.h declares; argument validation that happens on the host
returns status codes without touching a GPU."""
import ctypes

import pytest

from paper_1711_01897_gb300 import bem
from paper_1711_01897_gb300 import build as bem_build


@pytest.fixture(scope="module")
def lib():
    bem_build.build()
    return bem.load()


def test_exports_every_declared_function(lib):
    names = bem.header_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_text(lib):
    assert bem.bem_version() == 100
    assert isinstance(bem.bem_last_error(), str)


def test_host_side_argument_validation(lib):
    h = ctypes.c_void_p()
    assert lib.bem_mesh_create(None, 3, None, 1, ctypes.byref(h)) == 1
    assert lib.bem_mesh_create(None, 3, None, 1, None) == 1
    assert "null" in bem.bem_last_error()
    assert lib.bem_mesh_destroy(None) == 1
    assert lib.bem_mesh_size(None) == -1
    assert lib.bem_entries(None, 0, 0.0, 0, None, 1, None, 1, None, None) == 1
    assert lib.hmat_build_tree(None, 32, 1.2, ctypes.byref(h)) == 1
    assert lib.hmat_assemble(None, 0, 0.0, 1e-4, 0, None) == 1
    assert lib.hmat_matvec(None, None, None, 1, None) == 1
    assert lib.hmat_destroy(None) == 1
    assert lib.hmat_stats(None, None) == 1


def test_quadrature_class_arguments(lib):
    """bem_set_quadrature rejects negative and non-finite thresholds and keeps
    the previous ones; hmat_block_rules rejects null handles."""
    saved = bem.bem_get_quadrature()
    assert saved == {"rho3": 0.0, "rho1": 0.0}
    for bad in ((-1.0, 0.0), (0.0, -2.0), (float("nan"), 0.0), (float("inf"), 0.0)):
        with pytest.raises(bem.BemError):
            bem.bem_set_quadrature(*bad)
    assert bem.bem_get_quadrature() == saved
    bem.bem_set_quadrature(4.0, 12.0)
    assert bem.bem_get_quadrature() == {"rho3": 4.0, "rho1": 12.0}
    bem.bem_set_quadrature(0.0, 0.0)
    assert lib.bem_set_quadrature(None) == 1
    assert lib.hmat_block_rules(None, None, 0) == 1
