"""The C-ABI library loads and exports every symbol include/pa.h declares, and
argument validation rejects bad input before any device work (CPU only)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09025_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "pa_create" in names and "pa_anneal_step" in names and "pa_grad" in names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pa_[a-z0-9_]+)", out))
    assert set(names) <= exported


def _create(lib, D=3, L=4, kind=0, J=None, h=None, R=10, betas=(0.0, 1.0), n_sweeps=1, opt=None):
    import paper_1710_09025_gb300 as P
    P.load(lib._name)
    N = L ** D if L > 0 else 1
    if J is None:
        J = np.ones(D * max(N, 1), np.float32)
    J = np.ascontiguousarray(J, np.float32)
    b = np.ascontiguousarray(betas, np.float64)
    out = ctypes.c_void_p()
    hp = None if h is None else np.ascontiguousarray(h, np.float32).ctypes.data_as(ctypes.c_void_p)
    rc = P.load().pa_create(ctypes.byref(out), D, L, kind, J.ctypes.data_as(ctypes.c_void_p), hp, R,
                            b.ctypes.data_as(ctypes.c_void_p), len(b), n_sweeps, 1,
                            ctypes.byref(opt) if opt else None, None)
    return rc, out, P.pa_last_error(None)


@pytest.mark.parametrize("kw,needle", [
    (dict(D=4), "D must"), (dict(L=5), "even"), (dict(L=0), "even"), (dict(R=0), "R must"),
    (dict(betas=(0.5, 1.0)), "betas[0]"), (dict(betas=(0.0, 1.0, 0.5)), "non-decreasing"),
    (dict(betas=(0.0, float("nan"))), "finite"), (dict(n_sweeps=-1), "n_sweeps"),
    (dict(kind=0, J=np.full(192, 0.5, np.float32)), "exactly"),
    (dict(kind=1, J=np.full(192, 5000.0, np.float32)), "4096"),
    (dict(kind=1, J=np.full(192, np.nan, np.float32)), "NaN"),
    (dict(kind=0, h=np.full(64, 0.25, np.float32)), "no field"),
    (dict(kind=7), "kind"),
])
def test_validation_rejects(lib, kw, needle):
    rc, out, msg = _create(lib, **kw)
    assert rc == -1 and not out.value
    assert needle in msg


def test_option_validation(lib):
    import paper_1710_09025_gb300 as P
    P.load(lib._name)
    o = P.pa_options_default(accumulate_grad=1, separate_gather=1)
    rc, out, msg = _create(lib, kind=0, opt=o)
    assert rc != -1  # valid for +-J couplings too (no GPU here: the allocation fails instead)
    o = P.pa_options_default(rng_tag=16)
    rc, out, msg = _create(lib, opt=o)
    assert rc == -1 and "rng_tag" in msg
    o = P.pa_options_default(layout=1)
    rc, out, msg = _create(lib, kind=1, J=np.ones(192, np.float32) * 0.3, opt=o)
    assert rc == -1 and "packed" in msg


def test_resampling_option_validation(lib):
    import paper_1710_09025_gb300 as P
    P.load(lib._name)
    o = P.pa_options_default(resampling=2)
    rc, out, msg = _create(lib, opt=o)
    assert rc == -1 and "resampling" in msg
    o = P.pa_options_default(capacity=-1)
    rc, out, msg = _create(lib, opt=o)
    assert rc == -1 and "capacity" in msg
    o = P.pa_options_default(resampling=1, capacity=5)
    rc, out, msg = _create(lib, R=10, opt=o)
    assert rc == -1 and "capacity" in msg
    o = P.pa_options_default(populations=[10, 12])  # multinomial: at most R
    rc, out, msg = _create(lib, R=10, opt=o)
    assert rc == -1 and "populations" in msg
    o = P.pa_options_default(resampling=1, populations=[10, 200], capacity=100)
    rc, out, msg = _create(lib, R=10, opt=o)
    assert rc == -1 and "populations" in msg


def test_options_struct_matches_the_header(tmp_path):
    """ctypes' pa_options has the size and field offsets of the C struct."""
    import paper_1710_09025_gb300 as P
    names = [f[0] for f in P.pa_options._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pa.h"\nint main(void) {\n'
                   '  printf("%zu", sizeof(pa_options));\n' +
                   "".join(f'  printf(" %zu", offsetof(pa_options, {n}));\n' for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(P.pa_options)
    assert got[1:] == [getattr(P.pa_options, n).offset for n in names]


def test_workspace_size_is_positive_and_grows_with_R(lib):
    import paper_1710_09025_gb300 as P
    P.load(lib._name)
    a = P.pa_workspace_size(3, 8, 0, 1000, 11)
    b = P.pa_workspace_size(3, 8, 0, 100000, 11)
    assert 0 < a < b
    assert b % 256 == 0


def test_product_never_imports_or_links_the_oracle():
    pat = re.compile(r"(^\s*(from|import)\s+oracle\b)|liboracle|oracle\.h|\bor_(create|step|philox|spec|resample|exact)", re.M)
    for dp, _, fs in os.walk(os.path.join(ROOT, "paper_1710_09025_gb300")):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not pat.search(open(os.path.join(dp, f)).read()), f


def test_packed_sweep_parts_cover_every_lattice_once():
    """The packed sweep's lattice sizes are instantiated in four translation
    units; together they must list every supported (D, L) exactly once."""
    import re
    csrc = os.path.join(ROOT, "paper_1710_09025_gb300", "csrc")
    main = open(os.path.join(csrc, "pa_packed.cu")).read()
    block = main[main.index("#define PA_PACKED_CASES(X)"):main.index("bool packed_supported")]
    supported = re.findall(r"X\((\d), (\d+)\)", block)
    parts = []
    for k in range(4):
        src = open(os.path.join(csrc, f"pa_packed_part{k}.cu")).read()
        body = src[src.index("#define X(d, l)"):src.index("#undef X")]
        parts += re.findall(r"X\((\d), (\d+)\)", body.split("\n", 1)[1])
    assert len(parts) == len(set(parts))
    assert sorted(parts) == sorted(supported) and len(supported) == 17
