"""Writes airpf_exp_table.h: the constants of the table-driven double exponential of the FP64
path (Tang, "Table-driven implementation of the exponential function in IEEE floating-point
arithmetic", ACM TOMS 15(2), 1989): the 64 values 2^(j/64) rounded to double, 64 / ln 2,
and ln 2 / 64 split into a high part with 36 significant bits (so that n times it is exact
for |n| < 2^17) and the rest.  Computed with mpmath at 200 bits; run from this directory:
    python gen_exp_table.py > airpf_exp_table.h
"""
import mpmath

mpmath.mp.prec = 200


def hexd(v) -> str:
    return float(v).hex()


def main():
    ln2_64 = mpmath.log(2) / 64
    hi = mpmath.mpf(float(ln2_64))
    m, e = mpmath.frexp(hi)                     # keep 36 significant bits of the high part
    hi = mpmath.ldexp(mpmath.floor(mpmath.ldexp(m, 36)), e - 36)
    lo = ln2_64 - hi
    print("// Generated by gen_exp_table.py (the constants of the table-driven double exponential).")
    print("#pragma once")
    print("namespace airpf {")
    print(f"constexpr double kExpInvLn2x64 = {hexd(64 / mpmath.log(2))};   // 64 / ln 2")
    print(f"constexpr double kExpLn2d64Hi = {hexd(hi)};   // ln 2 / 64, 36 significant bits")
    print(f"constexpr double kExpLn2d64Lo = {hexd(lo)};   // ln 2 / 64 - kExpLn2d64Hi")
    print("__device__ const double kExp2Table[64] = {  // 2^(j/64), j = 0..63")
    vals = [hexd(mpmath.power(2, mpmath.mpf(j) / 64)) for j in range(64)]
    for i in range(0, 64, 4):
        print("    " + ", ".join(vals[i:i + 4]) + ",")
    print("};")
    print("}  // namespace airpf")


if __name__ == "__main__":
    main()
