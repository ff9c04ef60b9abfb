"""Writes airpf_sincos_table.h: the constants of the table-driven sine and cosine of 2 pi v
(v in [0, 1]) of the FP64 path's Box-Muller pairs: sin and cos of 2 pi j / 256 (j = 0..255)
rounded to double, and 2 pi / 256.  The method is the usual table-plus-polynomial one (as in
Tang's exponential and logarithm): 2 pi v = 2 pi j / 256 + x with |x| <= pi / 256, and the
angle-addition formulas with Taylor polynomials for sin x and cos x.  Computed with mpmath at
200 bits; run from this directory:
    python gen_sincos_table.py > airpf_sincos_table.h
"""
import mpmath

mpmath.mp.prec = 200


def hexd(v) -> str:
    # the zeros of sin and cos at multiples of pi / 2 are exact zeros (not 200-bit residues)
    return (0.0 if abs(v) < mpmath.mpf(2) ** -150 else float(v)).hex()


def table(name, vals, comment):
    print(f"__device__ const double {name}[256] = {{  // {comment}")
    for i in range(0, 256, 4):
        print("    " + ", ".join(hexd(v) for v in vals[i:i + 4]) + ",")
    print("};")


def main():
    ang = [2 * mpmath.pi * j / 256 for j in range(256)]
    print("// Generated by gen_sincos_table.py (the constants of the table-driven sine and cosine).")
    print("#pragma once")
    print("namespace airpf {")
    print(f"constexpr double kTwoPiDiv256 = {hexd(2 * mpmath.pi / 256)};   // 2 pi / 256")
    table("kSin256", [mpmath.sin(a) for a in ang], "sin(2 pi j / 256)")
    table("kCos256", [mpmath.cos(a) for a in ang], "cos(2 pi j / 256)")
    print("}  // namespace airpf")


if __name__ == "__main__":
    main()
