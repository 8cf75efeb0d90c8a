"""The library's elliptical-NFW expansion table (paper_2609_08649_b300/csrc/lf_cse_table.h,
written by the package's own generator) against the oracle's independent fit of the same
recipe (oracle/cse_nfw.py): the fitted profiles must agree over the fitted range, and the
float-float pairs must reproduce the FP64 values."""
import os
import re

import numpy as np

from oracle import cse_nfw as C

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2609_08649_b300", "csrc", "lf_cse_table.h")


def _list(txt, name):
    body = txt.split("#define " + name + " ")[1].split("#define")[0]
    return [float(t.rstrip("f")) for t in re.findall(r"[-+]?[0-9.]+e[-+][0-9]+f?", body)]


def test_table_matches_the_oracle_fit():
    txt = open(HDR).read()
    n = int(re.search(r"#define LF_CSE_N (\d+)", txt).group(1))
    s, a = np.array(_list(txt, "LF_CSE_S_LIST")), np.array(_list(txt, "LF_CSE_A_LIST"))
    so, ao = C.table()
    assert len(s) == len(a) == n == len(so)
    assert np.array_equal(s, so)                          # the same scales (and support)
    x = np.logspace(-4, 3, 7919)
    g_lib = (0.5 / (s[None] ** 2 + x[:, None] ** 2) ** 1.5) @ a
    assert np.abs(g_lib / C.g_approx(x) - 1).max() < 1e-12
    assert np.abs(g_lib / C.nfw_g(x).numpy() - 1).max() < 2e-6
    # the compiler rounds each float literal to the nearest float32
    f32 = lambda v: np.array(v).astype(np.float32).astype(np.float64)
    sff = f32(_list(txt, "LF_CSE_S_FF_LIST")).reshape(n, 2)
    cff = f32(_list(txt, "LF_CSE_C_FF_LIST")).reshape(n, 2)
    assert np.all(np.abs(sff.sum(1) / s - 1) < 2.0 ** -44)
    assert np.all(np.abs(cff.sum(1) / (a / s) - 1) < 2.0 ** -44)
