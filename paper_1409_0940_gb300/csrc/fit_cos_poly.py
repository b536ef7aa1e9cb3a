"""Fit the polynomial behind cos_rr() in common.cuh (run by hand; not part of the build).

After the reduction x = k pi + r, cos(x) = (-1)^k cos(r) with |r| <= pi/2, and
cos(r) is written as p(s), s = r^2, a polynomial of degree DEG in s.  Lawson's algorithm (iteratively reweighted least squares) drives the
least-squares fit on a dense grid of s towards the minimax one.  Prints the
float32 coefficients (constant term first), the fit error and the error of a
float32 Horner evaluation.
"""
import sys

import numpy as np

DEG = int(sys.argv[1]) if len(sys.argv) > 1 else 5


def main():
    s = np.linspace(0.0, (np.pi / 2) ** 2, 20001)
    f = np.cos(np.sqrt(s))
    V = np.vander(s, DEG + 1, increasing=True)
    w = np.ones_like(s)
    for _ in range(300):
        c, *_ = np.linalg.lstsq(V * np.sqrt(w)[:, None], f * np.sqrt(w), rcond=None)
        e = np.abs(V @ c - f)
        w = w * e
        w /= w.sum()
    c32 = c.astype(np.float32)
    s32 = s.astype(np.float32)
    p = np.full_like(s32, c32[-1])
    for k in range(DEG - 1, -1, -1):
        p = (p * s32 + c32[k]).astype(np.float32)
    print("coefficients:", [float(x) for x in c32])
    print("fit error %.3e, float32 evaluation error %.3e" % (np.abs(V @ c - f).max(), np.abs(p - f).max()))


if __name__ == "__main__":
    main()
