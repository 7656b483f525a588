"""Prints kExp2Tab of vrc_math64.h: 2^(j/256) for j = 0..255 as the nearest
float64 (head) and the nearest float64 to the remainder (tail), from exact
decimal arithmetic at 80 digits."""
from decimal import Decimal, getcontext


def exp2_table(n=256):
    getcontext().prec = 80
    ln2 = Decimal(2).ln()
    rows = []
    for j in range(n):
        v = (Decimal(j) / n * ln2).exp()
        hi = float(v)
        rows.append((hi, float(v - Decimal(hi))))
    return rows


if __name__ == "__main__":
    for hi, lo in exp2_table():
        print("    {%s, %s}," % (hi.hex(), lo.hex() if lo else "0x0p+0"))
