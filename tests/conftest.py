import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def tiny_inputs():
    """Tiny fixed-model survey: R band spectra (complex128), t_d, G_d (FP64)."""
    import synthetic as S
    s = S.tiny_survey()
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    return s, R, td, Gd


def small_survey(n=25, dx=20.0, nt=128, dt=0.008, nfocal=2, calibrate=0.7, fmax_hz=None, seed=3):
    """A small convergent survey on the tiny model (dense direct solve size)."""
    import synthetic as S
    from synthetic.layered import Survey
    base = S.tiny_survey()
    xs = [(n - 1) * dx / 2, (n - 1) * dx / 4, 3 * (n - 1) * dx / 4][:nfocal]
    zs = [650.0, 600.0, 700.0][:nfocal]
    return Survey("small", n=n, dx=dx, nt=nt, dt=dt, f0=20.0, fmax_hz=fmax_hz, model=base.model,
                  seed=seed, eps=0.024, focal=np.array(list(zip(xs, zs))), calibrate=calibrate)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
