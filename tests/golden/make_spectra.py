"""Writes spectra_examples.txt: spectral diagnostics of §3 (Figs. 1–2, Theorem GMRES) computed by
the oracle for Examples 1 and 2 at small N.  Calls only oracle/ and the input generators; run
`python tests/golden/make_spectra.py` from the repository root to regenerate."""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2404_10221_gb300 import workloads as W  # noqa: E402

CASES = [(1, (1.5,), 7), (1, (1.5,), 15), (1, (1.5,), 31), (1, (1.9,), 31), (2, (1.3, 1.5), 7)]
COLS = ["spread_A", "spread_PA", "re_PA_min", "re_PA_max", "v", "r", "sin_theta"]


def rows():
    out = []
    for d, alpha, n in CASES:
        wl = W.paper_example(d, list(alpha), n, 64)
        p, t = wl.prob, wl.field_tables()
        ebar, ehat, echeck = O.ebar_from_tables(p, t["e_tc"], t["e_sp"])
        e = O.eval_field_interior(p, t["e_tc"][0], t["e_sp"])
        s = O.spectral_summary(p, e, ebar)
        out.append((d, alpha, n, [s[c] for c in COLS], O.theorem_c(ehat, echeck)))
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "spectra_examples.txt"), "w") as fh:
        fh.write("# Spectral diagnostics (oracle, written by make_spectra.py): Examples 1-2 of §4 at M = 64,\n")
        fh.write("# step m = 0.  spread = max|lambda|/min|lambda| of Ã and of P^{-1}Ã; v, r: distance from 0 and\n")
        fh.write("# radius of the numerical range of P^{-1/2} Ã P^{-1/2}; sin_theta from Eq. (numrag);\n")
        fh.write("# c: the rate constant of Theorem GMRES.\n")
        fh.write("# d  alphas      N   " + "  ".join(COLS) + "  c\n")
        for d, alpha, n, vals, c in rows():
            a = ",".join("%.2f" % x for x in alpha)
            fh.write("%d  %-10s %3d  %s  %.12e\n" % (d, a, n, "  ".join("%.12e" % v for v in vals), c))
