"""Writes airpf_log_table.h: the constants of the table-driven double logarithm of the FP64
path (Tang, "Table-driven implementation of the logarithm function in IEEE floating-point
arithmetic", ACM TOMS 16(4), 1990): for F_j = 1 + j/128 (j = 0..128) the reciprocals 1/F_j
rounded to double and log F_j split into a high part on the grid 2^-42 and the rest, and
ln 2 split the same way, so that e ln2_hi + (log F_j)_hi is exact for |e| <= 1100.
Computed with mpmath at 200 bits; run from this directory:
    python gen_log_table.py > airpf_log_table.h
"""
import mpmath

mpmath.mp.prec = 200
GRID = mpmath.mpf(2) ** -42


def hexd(v) -> str:
    return float(v).hex()


def split(v):
    hi = mpmath.nint(v / GRID) * GRID
    return hi, v - hi


def table(name, vals, comment):
    print(f"__device__ const double {name}[129] = {{  // {comment}")
    for i in range(0, 129, 4):
        print("    " + ", ".join(hexd(v) for v in vals[i:i + 4]) + ",")
    print("};")


def main():
    F = [1 + mpmath.mpf(j) / 128 for j in range(129)]
    lhi, llo = split(mpmath.log(2))
    parts = [split(mpmath.log(f)) for f in F]
    print("// Generated by gen_log_table.py (the constants of the table-driven double logarithm).")
    print("#pragma once")
    print("namespace airpf {")
    print(f"constexpr double kLogLn2Hi = {hexd(lhi)};   // ln 2 on the grid 2^-42")
    print(f"constexpr double kLogLn2Lo = {hexd(llo)};   // ln 2 - kLogLn2Hi")
    table("kLogInvF", [1 / f for f in F], "1 / (1 + j/128)")
    table("kLogFHi", [h for h, _ in parts], "log(1 + j/128) on the grid 2^-42")
    table("kLogFLo", [lo for _, lo in parts], "log(1 + j/128) - kLogFHi[j]")
    print("}  // namespace airpf")


if __name__ == "__main__":
    main()
