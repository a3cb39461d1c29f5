"""The C-ABI library builds, loads and exports every symbol include/ppm.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ppm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w ]+\*?\s*\b(ppm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ppm_create", "ppm_build_grid", "ppm_gather_test_update", "ppm_radiance"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2504_04411_gb300 import build, ppm
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(ppm.EXPORTS) == _declared()


def test_default_params_and_strerror_without_gpu():
    from paper_2504_04411_gb300 import build, ppm
    build.build()
    p = ppm.ppm_default_params()
    assert p.k == pytest.approx(0.7) and p.alpha_f == pytest.approx(0.01)
    assert p.rmin_ratio == pytest.approx(1e-3) and p.cell_factor == 1.0
    assert ppm.ppm_strerror(ppm.PPM_ESTATE) == "call out of order"


def test_struct_layouts_match_header():
    from paper_2504_04411_gb300 import ppm
    # sizes implied by include/ppm.h on LP64
    assert ctypes.sizeof(ppm.ppm_hitpoints) == 48
    assert ctypes.sizeof(ppm.ppm_photons) == 64
    assert ctypes.sizeof(ppm.ppm_params) == 64
    assert ctypes.sizeof(ppm.ppm_iter_stats) == 64
    assert ctypes.sizeof(ppm.ppm_state_view) == 56
