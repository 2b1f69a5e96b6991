"""Shared helpers of the GPU tests, the smoke run and the bench (no oracle code)."""

from __future__ import annotations

import numpy as np

FIELD_NAMES = ["N", "f1plus", "f1min", "f2p", "pmin", "G"]


def desc_for(survey, rprec: int = 0, flags: int = 0, nfocal: int | None = None):
    from paper_2106_04649_gb300.api import Desc
    return Desc(nsrc=survey.n, nrec=survey.n, nt=survey.nt,
                nfocal=survey.nfocal if nfocal is None else nfocal, dt=survey.dt, dx=survey.dx,
                fmax_hz=survey.fmax_hz if survey.fmax_hz else 0.0, rprec=rprec, flags=flags)


def survey_inputs(survey, focal_idx=None, dtype=np.complex64):
    """(R band [nw][n][n], t_d [F][n], G_d [F][n][nt] float32) of a survey."""
    import synthetic as S
    R = S.reflection_band(survey, dtype=dtype)
    td = S.survey_td(survey)
    if focal_idx is not None:
        td = td[focal_idx]
    Gd = S.gd_traces(survey, td, np.float32)
    return R, td, Gd
