"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Calls only ``oracle/`` (and the seeded input generators).  Run from the repo
root: ``python tests/golden/make_golden.py``.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic as S  # noqa: E402
from oracle import marchenko as M  # noqa: E402


def main():
    s = S.tiny_survey()
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 16)
    e0 = float(np.sum(Gd ** 2))
    with open(os.path.join(HERE, "tiny_energy.txt"), "w") as f:
        f.write("# Tiny fixed-model survey (101 positions, nt=512, dt=4 ms, x_F=(500,650) m,\n")
        f.write("# eps=12 ms, full band), FP64 oracle: Algorithm 1 for 16 iterations.\n")
        f.write("# Columns: iteration i, E_i = sum N_i^2, sqrt(E_i / sum G_d^2).\n")
        f.write(f"# sum G_d^2 = {e0:.17e}\n")
        for i, e in enumerate(st.energy):
            f.write(f"{i} {float(e[0]):.17e} {np.sqrt(float(e[0]) / e0):.17e}\n")


if __name__ == "__main__":
    main()
