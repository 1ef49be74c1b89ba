"""Accuracy metrics (test infrastructure only).

* :func:`residual_fro` -- ||M X - I||_F / (||M||_F ||X||_F), the relative
  residual the accuracy targets are stated in.
* :func:`res_left`, :func:`res_right` -- the paper's left and right relative
  residuals in the max norm (Sec. 5.1, eq. "backerr"), with the complex max
  norm max(||Re||_max, ||Im||_max) (eq. "maxnorm").
* :func:`forward_error` -- ||X - X*||_max / ||X*||_max with the same norm.

Matrix products use numpy's matmul (a library primitive); no metric is
computed by the CUDA path.
"""
from __future__ import annotations

import numpy as np


def cmax(a) -> float:
    """Complex max norm (eq. "maxnorm"): max(||Re a||_max, ||Im a||_max)."""
    a = np.asarray(a)
    if a.size == 0:
        return 0.0
    if np.iscomplexobj(a):
        return float(max(np.abs(a.real).max(), np.abs(a.imag).max()))
    return float(np.abs(a).max())


def residual_fro(m, x) -> float:
    m = np.asarray(m, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    n = m.shape[0]
    r = m @ x - np.eye(n)
    return float(np.linalg.norm(r) / (np.linalg.norm(m) * np.linalg.norm(x)))


def res_right(m, x) -> float:
    m = np.asarray(m, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    return cmax(m @ x - np.eye(m.shape[0])) / (cmax(m) * cmax(x))


def res_left(m, x) -> float:
    m = np.asarray(m, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    return cmax(x @ m - np.eye(m.shape[0])) / (cmax(m) * cmax(x))


def forward_error(x, xstar) -> float:
    x = np.asarray(x, dtype=np.complex128)
    xstar = np.asarray(xstar, dtype=np.complex128)
    return cmax(x - xstar) / cmax(xstar)


def residual_cols(m, x, cols) -> float:
    """Max-norm residual of the sampled columns of M X - I, normalised like
    :func:`res_right`; for matrices too large for a full product."""
    m = np.asarray(m, dtype=np.complex128)
    cols = np.asarray(cols)
    xc = np.asarray(x, dtype=np.complex128)[:, cols]
    r = m @ xc
    r[cols, np.arange(len(cols))] -= 1.0
    return cmax(r) / (cmax(m) * cmax(xc))
