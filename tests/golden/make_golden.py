"""Write tests/golden/sin_pi_t.txt from the closed form in oracle.closed_form.

The paper's only worked example is x(t) = sin(pi t) on [0, 1] (Sec. 2,
Figs. 1 and 2), whose alpha-densified spectra it plots for several alpha
without printing values.  This script evaluates the closed form of Eq. 7
(scale S = T/N, T = 1) for that signal in 40-digit arithmetic and stores it to
17 significant digits.  It calls only the oracle package.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.closed_form import sin_pi_t_spectrum_mp  # noqa: E402

CASES = [(16, 16), (16, 32), (16, 64), (16, 128), (10, 25), (12, 8)]


def main():
    path = os.path.join(HERE, "sin_pi_t.txt")
    with open(path, "w") as f:
        f.write("# Closed-form Eq. 7 spectrum (S = T/N, T = 1) of x_n = sin(pi n/N), n < N:\n")
        f.write("# the worked example of Sec. 2 (Figs. 1-2: sin(pi t) sampled on [0, 1]).\n")
        f.write("# alpha = M/N in {1, 2, 4, 8, 2.5, 2/3}.  Columns: N M m Re(X_m) Im(X_m)\n")
        for N, M in CASES:
            vals = sin_pi_t_spectrum_mp(N, M)
            for m, (re, im) in enumerate(vals):
                f.write("%d %d %d %s %s\n" % (N, M, m, "%.17e" % float(re), "%.17e" % float(im)))
    print("wrote", path)


if __name__ == "__main__":
    main()
