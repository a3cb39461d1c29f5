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
    assert p.test == 0 and p.mapping == 0 and p.tile == 0 and p.wait_limit == 0
    assert list(p.reserved) == [0] * 3
    assert ppm.ppm_strerror(ppm.PPM_ESTATE) == "call out of order"
    assert ppm.ppm_strerror(ppm.PPM_ETIMEOUT) == "bounded device wait timed out"
    assert ppm.ppm_strerror(ppm.PPM_EINCOMPLETE).startswith("a gather skipped cells")


def test_struct_layouts_match_header():
    from paper_2504_04411_gb300 import ppm
    # sizes implied by include/ppm.h on LP64
    assert ctypes.sizeof(ppm.ppm_hitpoints) == 48
    assert ctypes.sizeof(ppm.ppm_photons) == 64
    assert ctypes.sizeof(ppm.ppm_params) == 64
    assert ctypes.sizeof(ppm.ppm_iter_stats) == 64
    assert ctypes.sizeof(ppm.ppm_state_view) == 56


def test_struct_field_offsets_match_the_header(tmp_path):
    """Every field of the binding's structs at the offset the C compiler
    gives it in include/ppm.h (a renamed, moved or resized field fails)."""
    import shutil
    import subprocess

    from paper_2504_04411_gb300 import ppm
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    names = ("ppm_hitpoints", "ppm_photons", "ppm_params", "ppm_iter_stats", "ppm_state_view")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ppm.h"', "int main(void)", "{"]
    for s in names:
        lines.append(f'    printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(ppm, s)._fields_:
            lines.append(f'    printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "offsets.c", tmp_path / "offsets"
    src.write_text("\n".join(lines) + "\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", str(src), "-o", str(exe),
                        "-I", os.path.join(root, "include")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s in names:
        cls = getattr(ppm, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"
