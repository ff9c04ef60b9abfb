"""The constants of the FP64 path's table-driven exponential and logarithm: the committed headers
are what their generators write; the exponential's table holds 2^(j/256) to the nearest double
and its split of ln 2 / 256 is exact when multiplied by any |n| < 2^19; the logarithm's table
holds 1/F_j to the nearest double and log F_j as an exact sum of a part on the grid 2^-42 and
the rest, with F_128 = 2 split like ln 2; the sine and cosine tables hold sin and cos of
2 pi j / 256, exact at the multiples of pi / 2."""
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2312_06484_gb300", "csrc")


def _header():
    return open(os.path.join(CSRC, "airpf_exp_table.h")).read()


def _consts(text):
    vals = {}
    for line in text.splitlines():
        if line.startswith("constexpr double"):
            name, v = line.split("constexpr double")[1].split(";")[0].split("=")
            vals[name.strip()] = float.fromhex(v.strip())
    start = text.index("{", text.index("kExp2Table")) + 1
    body = " ".join(ln.split("//")[0] for ln in text[start:text.index("}", start)].splitlines())
    table = [float.fromhex(t) for t in body.split(",") if t.strip()]
    return vals, table


def test_header_is_the_generator_output():
    pytest.importorskip("mpmath")
    out = subprocess.run([sys.executable, "gen_exp_table.py"], cwd=CSRC, capture_output=True, text=True, check=True)
    assert out.stdout == _header()


def test_table_and_split_constants():
    vals, table = _consts(_header())
    assert len(table) == 256
    for j, v in enumerate(table):
        # within an ulp of 2^(j/256) as exp2 gives it in double (itself within an ulp)
        assert abs(v - np.exp2(j / 256)) <= np.spacing(v)
    hi, lo = vals["kExpLn2dNHi"], vals["kExpLn2dNLo"]
    assert Fraction(hi).denominator.bit_length() <= 9 + 34 + 1        # 34 significant bits
    assert abs(hi + lo - np.log(2) / 256) < 1e-19
    n = 2 ** 19 - 1
    assert Fraction(n) * Fraction(hi) == Fraction(n * hi)               # n hi exact in double
    assert abs(vals["kExpInvLn2xN"] * np.log(2) / 256 - 1) < 3e-16


def _log_header():
    return open(os.path.join(CSRC, "airpf_log_table.h")).read()


def _log_tables(text):
    out = {}
    for name in ("kLogInvF", "kLogFHi", "kLogFLo"):
        start = text.index("{", text.index(name + "[129]")) + 1
        body = " ".join(ln.split("//")[0] for ln in text[start:text.index("}", start)].splitlines())
        out[name] = [float.fromhex(t) for t in body.split(",") if t.strip()]
    for line in text.splitlines():
        if line.startswith("constexpr double"):
            name, v = line.split("constexpr double")[1].split(";")[0].split("=")
            out[name.strip()] = float.fromhex(v.strip())
    return out


def test_log_header_is_the_generator_output():
    pytest.importorskip("mpmath")
    out = subprocess.run([sys.executable, "gen_log_table.py"], cwd=CSRC, capture_output=True, text=True, check=True)
    assert out.stdout == _log_header()


def test_log_tables():
    t = _log_tables(_log_header())
    grid = Fraction(1, 2 ** 42)
    for j in range(129):
        F = Fraction(128 + j, 128)
        inv = Fraction(t["kLogInvF"][j])
        assert abs(inv - 1 / F) <= Fraction(np.spacing(t["kLogInvF"][j])) / 2      # nearest double
        hi, lo = t["kLogFHi"][j], t["kLogFLo"][j]
        assert (Fraction(hi) / grid).denominator == 1                              # on the grid
        assert abs(hi + lo - np.log(float(F))) <= 2 * np.spacing(np.log(float(F)) or 1.0)
    assert t["kLogFHi"][128] == t["kLogLn2Hi"] and t["kLogFLo"][128] == t["kLogLn2Lo"]
    assert t["kLogFHi"][0] == 0.0 and t["kLogFLo"][0] == 0.0
    assert (Fraction(t["kLogLn2Hi"]) / grid).denominator == 1
    assert abs(t["kLogLn2Hi"] + t["kLogLn2Lo"] - np.log(2.0)) < 1e-17


def test_sincos_header_is_the_generator_output():
    pytest.importorskip("mpmath")
    out = subprocess.run([sys.executable, "gen_sincos_table.py"], cwd=CSRC, capture_output=True, text=True,
                         check=True)
    assert out.stdout == open(os.path.join(CSRC, "airpf_sincos_table.h")).read()


def test_sincos_tables():
    text = open(os.path.join(CSRC, "airpf_sincos_table.h")).read()
    tabs = {}
    for name in ("kSin256", "kCos256"):
        start = text.index("{", text.index(name + "[256]")) + 1
        body = " ".join(ln.split("//")[0] for ln in text[start:text.index("}", start)].splitlines())
        tabs[name] = np.array([float.fromhex(t) for t in body.split(",") if t.strip()])
    j = np.arange(256)
    assert np.abs(tabs["kSin256"] - np.sin(2 * np.pi * j / 256)).max() < 1e-15   # numpy rounds the angle
    assert np.abs(tabs["kCos256"] - np.cos(2 * np.pi * j / 256)).max() < 1e-15
    assert tabs["kSin256"][0] == 0 and tabs["kSin256"][128] == 0 and tabs["kSin256"][64] == 1
    assert tabs["kCos256"][64] == 0 and tabs["kCos256"][192] == 0 and tabs["kCos256"][128] == -1
    assert np.all(tabs["kSin256"][1:128] > 0) and np.all(tabs["kSin256"][129:] < 0)
