"""The C ABI library builds, loads without a GPU and exports what include/dsdna.h declares."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1608_03722_gb300 import _build, dsdna

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dsdna.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsdna_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = _build.build()
    names = declared_functions()
    assert len(names) >= 15
    L = C.CDLL(lib)
    for n in names:
        assert hasattr(L, n), n
    assert set(dsdna.EXPORTS) <= set(names)


def test_nm_lists_symbols_with_c_linkage():
    lib = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dsdna_[a-z_0-9]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_struct_layouts_match_the_header(tmp_path):
    """Compile a probe against the header and compare sizes/offsets with the ctypes mirrors."""
    probe = tmp_path / "probe.c"
    fields = {
        "dsdna_params": [f for f, _ in dsdna.dsdna_params._fields_],
        "dsdna_system": [f for f, _ in dsdna.dsdna_system._fields_],
        "dsdna_allocator": [f for f, _ in dsdna.dsdna_allocator._fields_],
        "dsdna_obs": [f for f, _ in dsdna.dsdna_obs._fields_],
        "dsdna_info": [f for f, _ in dsdna.dsdna_info._fields_],
        "dsdna_prof": [f for f, _ in dsdna.dsdna_prof._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(probe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, fs in fields.items():
        cls = getattr(dsdna, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_default_params_match_table_one():
    p = dsdna.dsdna_default_params()
    assert (p.K1, p.R0, p.sigma_bb, p.K2, p.rc_hb, p.K3, p.K4, p.lambda_m, p.r0_m, p.K5, p.K6) == \
        (30.0, 0.6825, 0.443, 6.0, 0.3, 50.0, 30.0, 8.0, 0.34, 200.0, 52.0)
    assert abs(p.d_dih * 180 / 3.141592653589793 + 144.0) < 1e-12
    assert p.dt == 0.005 and p.kT == 1.0 and p.ell == 0.5


def test_create_without_gpu_fails_cleanly():
    """No GPU here: create must return an error code, never crash or fall back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = dsdna.load()
    p = dsdna.dsdna_default_params()
    nb = (C.c_int * 1)(10)
    sys = dsdna.dsdna_system(1, nb, None, None, None, None, None)
    h = C.c_void_p()
    rc = L.dsdna_create(C.byref(p), C.byref(sys), None, None, C.byref(h))
    assert rc != 0 and not h.value
    assert L.dsdna_last_error(None)


@pytest.mark.parametrize("field,value", [("list_build", 2), ("list_build", -1), ("pair_halving", 2)])
def test_create_rejects_out_of_range_build_switches(field, value):
    """Parameter checks come before any device call, so they hold without a
    GPU: an out-of-range list_build or pair_halving is DSDNA_EINVAL, named in
    the error text."""
    L = dsdna.load()
    p = dsdna.dsdna_default_params()
    setattr(p, field, value)
    nb = (C.c_int * 1)(10)
    sys = dsdna.dsdna_system(1, nb, None, None, None, None, None)
    h = C.c_void_p()
    rc = L.dsdna_create(C.byref(p), C.byref(sys), None, None, C.byref(h))
    assert rc == -1 and not h.value, rc
    assert field in L.dsdna_last_error(None).decode()
