"""C-ABI boundary checks that need no GPU: the library builds, loads, exports every entry
point include/ebit.h declares, and rejects invalid configurations before touching the device."""
import os
import re
import subprocess

import pytest

from paper_2402_13677_gb300 import build as B
from paper_2402_13677_gb300 import ebit as E
from paper_2402_13677_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "ebit.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(ebit_[a-z_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ebit_init", "ebit_set_phase_props", "ebit_step", "ebit_get_field", "ebit_set_interface"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ebit_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)
        assert callable(getattr(E, n)), f"binding lacks {n}"


def test_version_string(lib):
    assert "sm_103a" in E.ebit_version()


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of the C structs have the C compiler's offsets and sizes."""
    import ctypes as C
    src = tmp_path / "layout.c"
    fields = [f[0] for f in E.ebit_config._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ebit.h"', "int main(void) {",
             '  printf("config %zu\\n", sizeof(ebit_config));',
             '  printf("props %zu\\n", sizeof(ebit_phase_props));',
             '  printf("alloc %zu\\n", sizeof(ebit_allocator));']
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof(ebit_config, {f}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(got["config"]) == C.sizeof(E.ebit_config)
    assert int(got["props"]) == C.sizeof(E.ebit_phase_props)
    assert int(got["alloc"]) == C.sizeof(E.ebit_allocator)
    for f in fields:
        assert int(got[f]) == getattr(E.ebit_config, f).offset, f


@pytest.mark.parametrize("mutate", [
    lambda c: setattr(c, "nx", 2),
    lambda c: setattr(c, "dt", -1.0),
    lambda c: setattr(c, "extend_iters", 1),
    lambda c: setattr(c, "precision", 7),
    lambda c: c.bc.__setitem__(0, 9),
    lambda c: setattr(c, "rtol", 0.0),
    lambda c: (setattr(c, "nx", 1 << 15), setattr(c, "ny", (1 << 14) + 2)),   # more than 2^29 cells
])
def test_init_rejects_invalid_config_without_device(lib, mutate):
    pb = w.stefan(16, 4, steps=0)
    c = E.config_from_problem(pb)
    mutate(c)
    with pytest.raises(E.EbitError) as ei:
        E.ebit_init([c])
    assert ei.value.status == E.EBIT_EINVAL


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    mod = importlib.import_module("paper_2402_13677_gb300.ebit")
    saved = mod._lib
    mod._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            mod.load(str(tmp_path / "missing.so"))
    finally:
        mod._lib = saved


def test_status_codes_match_the_header():
    """The binding's status numbers are the header's enum values."""
    hdr = open(os.path.join(ROOT, "include", "ebit.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    body = re.search(r"typedef enum \{(.*?)\} ebit_status;", hdr, flags=re.S).group(1)
    vals = {n: int(v) for n, v in re.findall(r"(EBIT_\w+)\s*=\s*(-?\d+)", body)}
    assert {v: n for n, v in vals.items()} == E.STATUS_NAMES
    for n, v in vals.items():
        assert getattr(E, n) == v


def test_solve_status_mapping(tmp_path):
    """A solve whose bounded device wait gave up is an error (EBIT_ECUDA) even when its residual
    looks converged; a non-finite residual is EBIT_ENONFINITE; otherwise converged or not.  The
    mapping both solve entry points use, compiled with the host compiler."""
    src = tmp_path / "status.cpp"
    src.write_text("\n".join([
        '#include <cstdio>',
        '#include "status.h"',
        "int main() {",
        "  for (int m = 0; m < 16; ++m)",
        '    std::printf("%d %d\\n", m, (int)ebit::solve_status(m & 1, m & 2, m & 4, m & 8));',
        "  return 0;",
        "}"]))
    exe = tmp_path / "status"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "paper_2402_13677_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True)
    got = dict(map(int, l.split()) for l in subprocess.run([str(exe)], capture_output=True,
                                                             text=True).stdout.splitlines())
    for m, s in got.items():
        cuda_ok, fault, nonfinite, converged = m & 1, m & 2, m & 4, m & 8
        if not cuda_ok or fault:
            assert s == E.EBIT_ECUDA, m        # a fault is never reported as success
        elif nonfinite:
            assert s == E.EBIT_ENONFINITE, m
        else:
            assert s == (E.EBIT_OK if converged else E.EBIT_ENOCONV), m
