"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every function include/kf.h declares.  Only host-side entry points that touch
no GPU are called here."""
import ctypes
import os
import re

import pytest

import paper_2105_01796_gb300 as kf
from paper_2105_01796_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(kf_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return kf.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("kf_fit", "kf_fit_ex", "kf_fit_host", "kf_create", "kf_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    handle = ctypes.CDLL(_build.LIB)
    missing = [n for n in declared_functions() if not hasattr(handle, n)]
    assert not missing, missing
    assert set(kf.EXPORTS) <= set(declared_functions())


def test_host_only_entry_points(lib):
    assert lib.kf_abi_version() == 4
    o = kf.kf_default_options()
    assert o.precision == 0 and abs(o.mass - 0.1056583755) < 1e-15
    assert o.h_max == 50.0 and o.n_iter == 3 and o.block == 128
    assert lib.kf_strerror(0) == b"success"
    assert lib.kf_strerror(-1) == b"invalid argument"
    # 90 doubles per state (FP64), 6 doubles + 54 floats (mixed)
    assert kf.kf_workspace_size(1000, 31, o) == 1000 * 31 * 720 + 256
    om = kf.kf_default_options(kf.KF_PRECISION_MIXED)
    assert kf.kf_workspace_size(1000, 31, om) == 1000 * 31 * (6 * 8 + 54 * 4) + 256
    # a workspace cap splits the batch into chunks
    oc = kf.kf_default_options(workspace_bytes=720 * 31 * 100)
    assert kf.kf_workspace_size(1000, 31, oc) == 100 * 31 * 720 + 256


def test_kernels_compiled_for_sm103a():
    # the build compiles every kernel for sm_103a only
    assert os.path.exists(_build.LIB)
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors have the C structs' sizes and field offsets (the
    header compiled with gcc on this host)."""
    import subprocess
    inc = os.path.join(os.path.dirname(__file__), "..", "include")
    checks = {
        "kf_tracks": kf.KfTracks, "kf_surfaces": kf.KfSurfaces, "kf_measurements": kf.KfMeasurements,
        "kf_field_map": kf.KfFieldMap, "kf_field": kf.KfField, "kf_material": kf.KfMaterial,
        "kf_outputs": kf.KfOutputs, "kf_options": kf.KfOptions,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kf.h"', "int main(void) {"]
    for cname, py in checks.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, py in checks.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)
