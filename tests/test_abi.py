"""The C-ABI library builds, loads, exports every symbol include/gpfvm.h
declares, and rejects invalid descriptors before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import gpfvm_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_05020_gb300 import build, gpfvm
    build.build()
    return gpfvm.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gpfvm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpfvm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2406_05020_gb300 import gpfvm
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in gpfvm.SIGNATURES, f"binding lacks {n}"


def test_strerror_and_version(lib):
    assert lib.gpfvm_strerror(-3).decode().startswith("IC/BC")
    assert "sm_103a" in lib.gpfvm_version().decode()


def _create(desc):
    from paper_2406_05020_gb300 import gpfvm
    h = C.c_void_p()
    return gpfvm.lib().gpfvm_create(C.byref(desc), 10, C.byref(h))


@pytest.mark.parametrize("mutate", [
    lambda d: setattr(d, "ndim", 4),
    lambda d: setattr(d, "n_terms", 0),
    lambda d: d.lengthscale.__setitem__(0, -1.0),
    lambda d: setattr(d, "outputscale", 0.0),
    lambda d: d.alpha[0].__setitem__(1, 3),
    lambda d: d.sets[0].order.__setitem__(0, 2),
    lambda d: setattr(d, "n_sets", 9),
    lambda d: setattr(d, "jitter", float("nan")),
])
def test_invalid_descriptors_rejected(lib, mutate):
    from paper_2406_05020_gb300 import gpfvm
    d, keep = gpfvm.make_desc(W.heat_2d(4, 4, 4, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2)))
    mutate(d)
    assert _create(d) == -1


def test_non_increasing_edges_rejected(lib):
    from paper_2406_05020_gb300 import gpfvm
    p = W.heat_1d(4, 4, n_ic=3, n_bc=2, pred=3)
    p.edges[1] = np.array([0.0, 0.5, 0.5, 0.7, 1.0])
    d, keep = gpfvm.make_desc(p)
    assert _create(d) == -1


def test_system_descriptor_fields(lib):
    """A system (Sec. 3.3) is passed with the equation and output of every term
    and the output of every set; a one-output problem leaves them unread."""
    from paper_2406_05020_gb300 import gpfvm
    d, keep = gpfvm.make_desc(W.shallow_water_2d(3, 4, 4, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2)))
    assert d.n_outputs == 3 and d.n_terms == 11
    assert list(d.term_eq)[:11] == [0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2]
    assert list(d.term_out)[:11] == [0, 1, 2, 1, 2, 0, 1, 2, 1, 0, 2]
    assert list(d.set_out)[:5] == [0, 1, 2, 1, 2]
    d1, keep1 = gpfvm.make_desc(W.heat_2d(4, 4, 4, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2)))
    assert d1.n_outputs == 0


@pytest.mark.parametrize("mutate", [
    lambda d: setattr(d, "n_outputs", 5),                    # above GPFVM_MAX_OUTPUTS
    lambda d: d.term_out.__setitem__(0, 3),                  # no such output
    lambda d: d.term_eq.__setitem__(3, 5),                   # a gap in the equation numbers
    lambda d: d.set_out.__setitem__(1, -1),                  # no such output for a set
])
def test_invalid_system_descriptors_rejected(lib, mutate):
    from paper_2406_05020_gb300 import gpfvm
    d, keep = gpfvm.make_desc(W.shallow_water_2d(3, 4, 4, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2)))
    mutate(d)
    assert _create(d) == -1


def test_system_with_coefficient_field_rejected(lib):
    """Systems take constant coefficients: a coefficient field is refused."""
    from paper_2406_05020_gb300 import gpfvm
    p = W.wave_1d_system(3, 4, pred=(2, 2))
    p.fields = [None, np.ones(p.N // 2), None, None]
    d, keep = gpfvm.make_desc(p)
    assert _create(d) == -1


def test_binding_checks_system_lists():
    """The binding refuses per-term lists of the wrong length and too many outputs."""
    from dataclasses import replace

    from paper_2406_05020_gb300 import gpfvm
    p = W.wave_1d_system(3, 4, pred=(2, 2))
    with pytest.raises(ValueError):
        gpfvm.make_desc(replace(p, term_out=[0, 1, 1]))
    with pytest.raises(ValueError):
        gpfvm.make_desc(replace(p, n_out=5))
