"""Writes g_rationals.txt: Eq. 3 of the paper evaluated in exact rational
arithmetic at a few xi (the nested form exactly as printed, zeta = max(0,xi-1)).
Run: python tests/golden/make_g_rationals.py"""
import os
from fractions import Fraction as F


def g_exact(xi: F) -> F:
    if xi > 2:
        return F(0)
    zeta = max(F(0), xi - 1)
    inner = F(-8, 5) + xi ** 2 * (F(8, 5) + xi * (F(-1, 2) + xi * (F(-12, 35) + xi * F(3, 20))))
    return 1 + xi ** 3 * inner - zeta ** 6 * (F(3, 35) + xi * (F(18, 35) + xi * F(1, 5)))


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "g_rationals.txt")
    with open(out, "w") as f:
        f.write("# Eq. 3 (cutoff function g_P3M, Sec. II) in exact rational arithmetic\n")
        f.write("# xi_num xi_den g_num g_den\n")
        for xi in [F(0), F(1, 4), F(1, 2), F(3, 4), F(1), F(5, 4), F(3, 2), F(7, 4), F(2), F(9, 4)]:
            g = g_exact(xi)
            f.write(f"{xi.numerator} {xi.denominator} {g.numerator} {g.denominator}\n")
