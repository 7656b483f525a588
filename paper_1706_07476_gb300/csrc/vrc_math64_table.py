"""Writes vrc_exp2_table.h, the table kExp2Tab of vrc_math64.h: 2^(j/2048) for
j = 0..2047 as the nearest float64 (head) and the nearest float64 to the
remainder (tail), from exact decimal arithmetic at 80 digits.

    python vrc_math64_table.py > vrc_exp2_table.h
"""
from decimal import Decimal, getcontext

N = 2048


def exp2_table(n=N):
    getcontext().prec = 80
    ln2 = Decimal(2).ln()
    rows = []
    for j in range(n):
        v = (Decimal(j) / n * ln2).exp()
        hi = float(v)
        rows.append((hi, float(v - Decimal(hi))))
    return rows


if __name__ == "__main__":
    print("// 2^(j/%d), j = 0..%d: the nearest float64 and the nearest float64 to the" % (N, N - 1))
    print("// remainder.  Written by vrc_math64_table.py (exact decimal arithmetic);")
    print("// included by vrc_math64.h only.")
    print("#pragma once")
    print()
    print("#ifdef __CUDACC__")
    print("__device__")
    print("#endif")
    print("static const double kExp2Tab[%d][2] = {" % N)
    for hi, lo in exp2_table():
        print("    {%s, %s}," % (hi.hex(), lo.hex() if lo else "0x0p+0"))
    print("};")
