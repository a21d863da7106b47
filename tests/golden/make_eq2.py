"""Writes eq2_mixture.txt: the paper's closed-form entropy of the toy mixture
(Sec. 2.1, Eq. 2) evaluated at 60-digit precision with mpmath.

Each row is M, n0, n1: a window whose background (delta at one intensity)
contributes n0 voxels and whose salient part spreads n1 voxels on each of
the M bins, one of which coincides with the background bin.  Then
N = n0 + M*n1 and alpha = M*n1/N, and Eq. 2 gives
  H(alpha) = -(alpha/M + 1 - alpha) ln(alpha/M + 1 - alpha)
             - alpha (M-1)/M ln(alpha/M).
"""
import os

import mpmath as mp

mp.mp.dps = 60
ROWS = [(M, n0, n1) for M in (2, 4, 16, 64) for n0, n1 in
        ((0, 1), (1, 1), (5, 3), (100, 1), (7, 50), (1000, 17), (3, 2000))]


def eq2(M, alpha):
    M = mp.mpf(M)
    a = mp.mpf(alpha)
    g = a / M + 1 - a
    h = -(g * mp.log(g))
    if a > 0:
        h -= a * (M - 1) / M * mp.log(a / M)
    return h


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eq2_mixture.txt")
    with open(out, "w") as f:
        f.write("# Eq. 2 (Sec. 2.1) of arXiv 1310.6736 at 60 digits; columns: M n0 n1 H\n")
        for M, n0, n1 in ROWS:
            N = n0 + M * n1
            alpha = mp.mpf(M * n1) / N
            f.write(f"{M} {n0} {n1} {mp.nstr(eq2(M, alpha), 30)}\n")


if __name__ == "__main__":
    main()
