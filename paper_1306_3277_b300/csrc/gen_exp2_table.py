"""Writes pf_exp2_table.h: 2^(j/256), j = 0..255, each rounded to the nearest
double (computed with 80 decimal digits), for the table-driven weight
exponential of the propagate kernels (Tang, ACM TOMS 15(2), 1989).

    python gen_exp2_table.py > pf_exp2_table.h
"""
import mpmath

mpmath.mp.dps = 80


def nearest_double(v):
    # mpmath rounds to the nearest double when converting from 80 digits
    return float(mpmath.mpf(v))


def main():
    vals = [nearest_double(mpmath.power(2, mpmath.mpf(j) / 256)) for j in range(256)]
    print("// Generated by gen_exp2_table.py: 2^(j/256), j = 0..255, nearest double.")
    print("#pragma once")
    print("static __device__ double k_exp2_256[256] = {")
    for r in range(0, 256, 4):
        print("    " + ", ".join(v.hex() for v in vals[r:r + 4]) + ",")
    print("};")


if __name__ == "__main__":
    main()
