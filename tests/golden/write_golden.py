"""Writes the closed-form fixture of the Gaussian covariance square root.

For a Gaussian correlation exp(-d^2 / (2 L^2)) on an infinite line, the
square root under convolution is sigma_b (2 / (pi L^2))^{1/4} exp(-d^2 / L^2).
On a circle of n >> L points the discrete circulant square root differs from
it by aliasing terms of order exp(-pi^2 L^2), far below FP64 rounding for
L >= 2.  Uses no oracle code.
"""
import os

import numpy as np


def main():
    L, sigma_b = 2.0, 1.0
    d = np.arange(0, 14)
    taps = sigma_b * (2.0 / (np.pi * L * L)) ** 0.25 * np.exp(-(d * d) / (L * L))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "gaussian_taps_closed_form.txt")
    with open(path, "w") as f:
        f.write("# d  tap  (sigma_b=1, L=2; continuous-limit closed form)\n")
        for di, t in zip(d, taps):
            f.write("%d %.17e\n" % (di, t))


if __name__ == "__main__":
    main()
