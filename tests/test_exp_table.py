"""The constants of the device exponential (Tang's table-driven method, 64 entries): every
table entry is 2^(j/64) rounded to the nearest double, the head of ln2/64 has at most 29
significant bits (its product with the reduction integer is exact) and head + tail equals
ln2/64 to far below a double's precision; all checked against 60-digit values."""
import os
import re

import pytest

mpmath = pytest.importorskip("mpmath")

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2011_07632_gb300", "csrc", "common.cuh")


def _source():
    return open(SRC).read()


def test_table_entries_are_rounded_powers_of_two():
    s = _source()
    body = s[s.index("EXP2_TABLE_BEGIN"):s.index("EXP2_TABLE_END")]
    vals = [float.fromhex(t) for t in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == 64
    mpmath.mp.dps = 60
    for j, v in enumerate(vals):
        exact = mpmath.power(2, mpmath.mpf(j) / 64)
        assert v == float(exact), j            # mpmath -> float rounds to nearest


def test_reduction_constants():
    s = _source()
    get = lambda name: float.fromhex(re.search(name + r" = (-?0x[0-9a-f.]+p[+-]\d+)", s).group(1))
    inv, hi, lo = get("kInvStep"), get("kStepHi"), get("kStepLo")
    mpmath.mp.dps = 60
    step = mpmath.log(2) / 64
    assert inv == float(1 / step)
    m, e = mpmath.frexp(mpmath.mpf(hi))
    assert (m * 2 ** 29) == int(m * 2 ** 29)   # at most 29 significant bits
    assert abs(mpmath.mpf(hi) + mpmath.mpf(lo) - step) < mpmath.mpf(2) ** -95
