"""The Taylor tables of J0, J1, Y0, Y1 that the fill uses for real arguments
in [4, 64) (csrc/mlqp_bessel_taylor.inc), evaluated on the CPU the way the
kernel does (Horner about the centre of the argument's half-unit interval)
and compared with 30-digit mpmath values on a sweep that includes every
interval's ends: within 3e-16 absolute (SciPy's own Y0 is off by up to
1.4e-15 near x = 5, so it is not the reference here)."""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

INC = os.path.join(os.path.dirname(__file__), "..", "paper_1410_5003_gb300", "csrc", "mlqp_bessel_taylor.inc")


def table():
    text = open(INC).read()
    deg = int(re.search(r"BESSEL_TAYLOR_DEG = (\d+);", text).group(1))
    body = text[text.index("{") + 1:text.rindex("}")]
    vals = np.array([float(v) for v in body.replace("\n", " ").split(",") if v.strip()])
    nc = deg + 1
    return vals.reshape(-1, 4, nc), nc


def evaluate(x, tab, nc):
    m = np.minimum(((x - 4.0) * 2.0).astype(int), tab.shape[0] - 1)
    t = x - (4.25 + 0.5 * m)
    out = []
    for f in range(4):
        c = tab[m, f]
        a = c[:, nc - 1].copy()
        for k in range(nc - 2, -1, -1):
            a = a * t + c[:, k]
        out.append(a)
    return out


def test_taylor_tables_match_mpmath():
    tab, nc = table()
    assert tab.shape[0] == 120
    rng = np.random.default_rng(11)
    x = np.concatenate([4.0 + 0.5 * np.arange(120), 4.5 + 0.5 * np.arange(119) - 1e-12, rng.uniform(4.0, 64.0, 600)])
    got = evaluate(x, tab, nc)
    mp.mp.dps = 30
    for f, (fn, n) in enumerate(((mp.besselj, 0), (mp.besselj, 1), (mp.bessely, 0), (mp.bessely, 1))):
        ref = np.array([float(fn(n, mp.mpf(float(v)))) for v in x])
        assert np.max(np.abs(got[f] - ref)) < 3e-16, (f, float(np.max(np.abs(got[f] - ref))))
