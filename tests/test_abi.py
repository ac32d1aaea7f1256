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


def _struct_fields(name):
    """(type, field) pairs of a typedef struct in include/dogip.h, comments removed."""
    src = open(os.path.join(ROOT, "include", "dogip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if decl:
            typ, names = re.match(r"(\w+)\s+(.*)", decl).groups()
            out += [(typ, nm.strip()) for nm in names.split(",")]
    return out


def test_solve_opts_layout_and_defaults(lib):
    """The binding's ctypes mirror of dogip_solve_opts has the header's fields in the
    header's order and types (an ABI drift would scramble every solve option), and
    dogip_solve_opts_default fills the documented defaults."""
    ctype = {"int": C.c_int, "double": C.c_double}
    hdr = _struct_fields("dogip_solve_opts")
    py = lib.SolveOpts._fields_
    assert [f for _, f in hdr] == [f for f, _ in py]
    assert all(ctype[t] is pt for (t, _), (_, pt) in zip(hdr, py))
    o = lib.SolveOpts()
    assert lib.lib.dogip_solve_opts_default(C.byref(o)) == lib.OK
    assert o.mode == lib.SOLVE_FP64 and o.tol == 1e-8 and o.check_every == 16
    assert o.inner_tol == 1e-4 and o.reliable_delta == 0.1 and o.scatter == -1
    assert o.inner_prec == lib.FP32 and o.inner_recurrence == 0 and o.single_launch == -1


def test_solve_info_layout(lib):
    hdr = _struct_fields("dogip_solve_info")
    assert [f for _, f in hdr] == [f for f, _ in lib.SolveInfo._fields_]


@pytest.mark.parametrize("cname,pyname", [("dogip_opts", "Opts"), ("dogip_info", "Info")])
def test_setup_struct_layouts(lib, cname, pyname):
    ctype = {"int": C.c_int, "double": C.c_double, "int64_t": C.c_int64}
    hdr = _struct_fields(cname)
    py = getattr(lib, pyname)._fields_
    assert [f for _, f in hdr] == [f for f, _ in py]
    assert all(ctype[t] is pt for (t, _), (_, pt) in zip(hdr, py))
