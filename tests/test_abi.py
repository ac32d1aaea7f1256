"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/dogip.h declares, rejects invalid input before touching the device, and
its compiled reference tables equal the oracle's exact tables."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "dogip.h")).read()
    return sorted(set(re.findall(r"^DOGIP_API\s+[\w\s\*]*?\b(dogip_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("dogip_setup", "dogip_apply", "dogip_solve", "dogip_destroy", "dogip_grad_coef",
                 "dogip_set_coef", "dogip_load", "dogip_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib.lib, n)]
    assert not missing, missing


def test_version_and_error_string(lib):
    assert lib.lib.dogip_version() >= 100
    assert isinstance(lib.lib.dogip_last_error(), bytes)


@pytest.mark.parametrize("d,p,form", [(2, p, f) for p in range(1, 9) for f in ("projection", "elliptic")]
                         + [(3, p, f) for p in (1, 2, 3, 4) for f in ("projection", "elliptic")])
def test_tables_equal_oracle(lib, d, p, form):
    """B and w of the library (compiled into the kernels for p <= 4 (3D: 3), run-time
    tables above) == the oracle's exact rationals rounded once, bit for bit."""
    from oracle import refelem
    B, w = lib.get_tables(d, p, form)
    ref = refelem.bhat(form, d, p)
    if form == "projection":
        ref = ref[None]
    assert B.shape == ref.shape
    assert np.array_equal(B, ref)
    assert np.array_equal(w, refelem.what(d, refelem.w_degree(form, p)))


def test_unsupported_order(lib):
    sizes = (C.c_int * 3)()
    assert lib.lib.dogip_get_tables(3, 5, 1, None, None, sizes) == lib.EUNSUPPORTED
    assert lib.lib.dogip_get_tables(2, 9, 1, None, None, sizes) == lib.EUNSUPPORTED


def test_setup_rejects_bad_input_on_host(lib):
    """Argument checks run before any CUDA call (dim, form, empty mesh, vertex ids)."""
    from paper_1710_09913_gb300 import inputs
    coords, cells = inputs.lattice_mesh(2, 2)
    coef = np.ones(len(cells))
    with pytest.raises(lib.DogipError) as e:
        lib.Context(np.zeros((4, 4)), cells, 1, "elliptic", coef)
    assert e.value.code == lib.EINVAL
    bad = cells.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(lib.DogipError) as e:
        lib.Context(coords, bad, 1, "elliptic", coef)
    assert e.value.code == lib.EINVAL
    with pytest.raises(lib.DogipError) as e:
        lib.Context(coords, cells, 1, "projection", np.ones((len(cells), 2, 2)))
    assert e.value.code == lib.EINVAL
    with pytest.raises(lib.DogipError) as e:
        lib.Context(coords, cells, 0, "elliptic", coef)
    assert e.value.code == lib.EINVAL
    nanc = coords.copy()
    nanc[3, 1] = np.nan
    with pytest.raises(lib.DogipError) as e:
        lib.Context(nanc, cells, 1, "elliptic", coef)
    assert e.value.code == lib.EINVAL
