"""The autotuner's JSON cache (gxp_tune_cache_get / _put): host-only calls,
so this runs without a GPU. A record written is read back exactly, the file
is valid JSON with one member per key, a key can be replaced, and a missing
key or file is reported."""
import ctypes as C
import json

import pytest

from paper_2203_13005_gb300 import gxp


def _rec(**kw):
    r = gxp.gxp_tune_record()
    for k, v in kw.items():
        setattr(r, k, v)
    return r


def test_tune_cache_round_trip(tmp_path):
    lib = gxp.load()
    path = str(tmp_path / "tune.json").encode()
    key1 = b"sssp_batch V=16777216 E=268435456 deg=4 esize=4 gpu=NVIDIA GB300"
    key2 = b"sssp_batch V=4096 E=65536 deg=4 esize=8 gpu=NVIDIA GB300"
    out = gxp.gxp_tune_record()
    assert lib.gxp_tune_cache_get(path, key1, C.byref(out)) == gxp.GXP_E_INVAL   # no file yet
    r1 = _rec(k1=1.25e-7, k2=3.1e-8, k3=0.0, a=0.0123, model_block_edges=3.5e7, block_edges=38347923.0,
              sweep_best_ms=8.75)
    assert lib.gxp_tune_cache_put(path, key1, C.byref(r1)) == gxp.GXP_OK
    r2 = _rec(k1=2.0, k2=3.0, k3=4.0, a=5.0, model_block_edges=6.0, block_edges=7.0, sweep_best_ms=8.0)
    assert lib.gxp_tune_cache_put(path, key2, C.byref(r2)) == gxp.GXP_OK
    assert lib.gxp_tune_cache_get(path, key1, C.byref(out)) == gxp.GXP_OK
    for f, _ in gxp.gxp_tune_record._fields_:
        assert getattr(out, f) == getattr(r1, f), f     # 17 significant digits: exact
    data = json.loads(open(path).read())
    assert set(data) == {key1.decode(), key2.decode()}
    assert data[key2.decode()]["block_edges"] == 7.0
    # replace one member, keep the other
    r2.block_edges = 9.0
    assert lib.gxp_tune_cache_put(path, key2, C.byref(r2)) == gxp.GXP_OK
    data = json.loads(open(path).read())
    assert len(data) == 2 and data[key2.decode()]["block_edges"] == 9.0
    assert lib.gxp_tune_cache_get(path, b"sssp_batch V=1 E=1", C.byref(out)) == gxp.GXP_E_INVAL
    assert lib.gxp_tune_cache_get(None, key1, C.byref(out)) == gxp.GXP_E_INVAL
    assert lib.gxp_tune_cache_put(str(tmp_path / "no" / "dir.json").encode(), key1, C.byref(r1)) == gxp.GXP_E_INVAL
