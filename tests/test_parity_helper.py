"""The parity comparison itself, on CPU: oracle output converted to the AOV
layout must compare as identical, and planted differences must be caught."""
import numpy as np

import scenes
from parity import AGREE_MIN, compare

AOV_DTYPE = np.dtype([("t", "<f4"), ("inst", "<u4"), ("geom", "<u4"), ("prim", "<u4"), ("n", "<f4", 3),
                      ("flags", "<u4"), ("refl_t", "<f4"), ("refl_inst", "<u4"), ("refl_geom", "<u4"),
                      ("refl_prim", "<u4")])


def _as_aov(ref):
    a = np.zeros(len(ref), AOV_DTYPE)
    for k in ("t", "refl_t"):
        a[k] = ref[k]
    for k in ("inst", "geom", "prim", "refl_inst", "refl_geom", "refl_prim"):
        a[k] = np.where(ref[k] < 0, 0xFFFFFFFF, ref[k].astype(np.int64)).astype(np.uint32)
    a["n"] = ref["n"]
    a["flags"] = ref["flags"] & 31
    return a


def test_compare_identity_and_planted_differences(oracle_lib):
    w = scenes.teaser(width=96, height=54)
    ref = oracle_lib.render(w)
    a = _as_aov(ref)
    rgb = ref["rgb"].astype(np.float32)
    rep = compare(ref, a, rgb, 50.0)
    assert rep["agree"] == 1.0 and rep["t_bad"] == rep["n_bad"] == rep["rgb_bad"] == 0
    hit = np.nonzero(ref["flags"] & 1)[0]
    b = a.copy()
    b["inst"][hit[:10]] += 1
    assert compare(ref, b, rgb, 50.0)["n_disagree"] == 10
    c = a.copy()
    c["t"][hit[0]] += 1.0
    assert compare(ref, c, rgb, 50.0)["t_bad"] == 1
    d = rgb.copy()
    d[hit[1]] += 0.01
    assert compare(ref, a, d, 50.0)["rgb_bad"] == 1
    e = a.copy()
    e["flags"][hit[2]] ^= 4
    assert compare(ref, e, rgb, 50.0)["agree"] < 1.0
    assert AGREE_MIN == 0.999
