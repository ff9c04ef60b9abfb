"""Writes airpf_exp_table.h: the constants of the table-driven double exponential of the FP64
path (Tang, "Table-driven implementation of the exponential function in IEEE floating-point
arithmetic", ACM TOMS 15(2), 1989): the 256 values 2^(j/256) rounded to double, 256 / ln 2,
and ln 2 / 256 split into a high part with 34 significant bits (so that n times it is exact
for |n| < 2^19) and the rest.  Computed with mpmath at 200 bits; run from this directory:
    python gen_exp_table.py > airpf_exp_table.h
"""
import mpmath

mpmath.mp.prec = 200


def hexd(v) -> str:
    return float(v).hex()


def main():
    ln2_n = mpmath.log(2) / 256
    hi = mpmath.mpf(float(ln2_n))
    m, e = mpmath.frexp(hi)                     # keep 34 significant bits of the high part
    hi = mpmath.ldexp(mpmath.floor(mpmath.ldexp(m, 34)), e - 34)
    lo = ln2_n - hi
    print("// Generated by gen_exp_table.py (the constants of the table-driven double exponential).")
    print("#pragma once")
    print("namespace airpf {")
    print(f"constexpr double kExpInvLn2xN = {hexd(256 / mpmath.log(2))};   // 256 / ln 2")
    print(f"constexpr double kExpLn2dNHi = {hexd(hi)};   // ln 2 / 256, 34 significant bits")
    print(f"constexpr double kExpLn2dNLo = {hexd(lo)};   // ln 2 / 256 - kExpLn2dNHi")
    print("__device__ const double kExp2Table[256] = {  // 2^(j/256), j = 0..255")
    vals = [hexd(mpmath.power(2, mpmath.mpf(j) / 256)) for j in range(256)]
    for i in range(0, 256, 4):
        print("    " + ", ".join(vals[i:i + 4]) + ",")
    print("};")
    print("}  // namespace airpf")


if __name__ == "__main__":
    main()
