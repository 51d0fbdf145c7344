"""The table of the kernels' weight exponential (Tang's method: 2^(j/256),
j = 0..255): every entry is the nearest double to 2^(j/256), and the committed
header is what its generator writes."""
import os
import re
import subprocess
import sys

import mpmath

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1306_3277_b300", "csrc")


def _entries(text):
    return [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", text)]


def test_table_entries_are_nearest_doubles():
    mpmath.mp.dps = 60
    vals = _entries(open(os.path.join(CSRC, "pf_exp2_table.h")).read())
    assert len(vals) == 256 and vals[0] == 1.0
    for j, v in enumerate(vals):
        exact = mpmath.power(2, mpmath.mpf(j) / 256)
        ulp = mpmath.mpf(2) ** (mpmath.floor(mpmath.log(exact, 2)) - 52)
        assert abs(mpmath.mpf(v) - exact) <= ulp / 2, j


def test_header_matches_generator():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp2_table.py")],
                         capture_output=True, text=True, check=True).stdout
    assert out == open(os.path.join(CSRC, "pf_exp2_table.h")).read()
