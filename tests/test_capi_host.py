"""Host-side checks of libgxp.so that need no GPU: it loads, exports every
symbol include/gxp.h declares, and its host-only block-size model agrees with
the oracle's Lemma 1."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import lemma1 as L
from paper_2203_13005_gb300 import gxp

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "gxp.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"GXP_API\s+[\w\s\*]+?\b(gxp_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = gxp.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # and the binding knows them all with a signature
    assert set(names) <= {n for n, _, _ in gxp.SIGNATURES}


def test_status_strings():
    lib = gxp.load()
    assert lib.gxp_status_string(0) == b"GXP_OK"
    assert lib.gxp_status_string(6) == b"GXP_E_STATE"


def test_null_handles_rejected():
    lib = gxp.load()
    assert lib.gxp_superstep(None, 0, 0, 0, 0, None) == gxp.GXP_E_INVAL
    assert lib.gxp_init(0, None, None) == gxp.GXP_E_INVAL
    lib.gxp_destroy(None)


def _cases():
    rng = np.random.default_rng(7)
    out = [(*L.PAPER_COEFFS[k], d) for k in L.PAPER_COEFFS for d in (117_180_000, 1 << 26, 1 << 28)]
    for _ in range(40):
        k = rng.uniform(0.01, 1.0, 3)
        out.append((float(k[0]), float(k[1]), float(k[2]), float(10 ** rng.uniform(0, 5)),
                    int(10 ** rng.uniform(3, 8))))
    return out


@pytest.mark.parametrize("k1,k2,k3,a,d", _cases())
def test_block_size_model_matches_lemma1(k1, k2, k3, a, d):
    b, s, t = gxp.block_size_model(k1, k2, k3, a, d)
    bo, so, to = L.lemma1_integer(k1, k2, k3, a, d)
    assert s == so
    assert t == pytest.approx(to, rel=1e-12)
    assert b == int(np.ceil(bo - 1e-9))


def test_block_size_model_rejects_bad_input():
    with pytest.raises(gxp.GxpError):
        gxp.block_size_model(0.1, 0.2, 0.3, 10.0, 1)


def test_init_without_gpu_reports_error():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(gxp.GxpError) as ei:
        gxp.Context(0)
    assert ei.value.code in (gxp.GXP_E_CUDA, gxp.GXP_E_INVAL)


def test_binding_structs_match_the_header(tmp_path):
    # every struct of the ABI: the C compiler's size and field offsets equal
    # the ctypes binding's
    import ctypes as C
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [gxp.gxp_config, gxp.gxp_stats, gxp.gxp_batch_opts, gxp.gxp_batch_report, gxp.gxp_serve_opts,
               gxp.gxp_query_info, gxp.gxp_serve_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gxp.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == C.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)
