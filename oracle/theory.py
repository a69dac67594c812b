"""Large-system analysis of PD/FD linear equalizers (closed forms and fixed points).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

All quantities use the paper's normalization: Rayleigh entries CN(0, 1/B)
(Def. 2), system ratio ``beta = U/B`` (Def. 1), ``snr = Es/N0`` in that
normalization.  With the generator's CN(0, 1) channels the same system has
``Es/N0_paper = B * Es / N0``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["psi", "fixed_point", "sinr_pd", "sinr_fd_lmmse", "sinr_fd_lmmse_uniform",
           "sinr_fd_zf", "message_entries", "db"]


def db(x):
    return 10.0 * np.log10(x)


def psi(kind: str, s2: float, Es: float) -> float:
    """MSE functions of Thm. 1: MRC ``Es``, ZF ``sigma^2``, L-MMSE ``Es sigma^2 / (Es + sigma^2)``."""
    if kind == "mrc":
        return Es
    if kind == "zf":
        return s2
    if kind == "lmmse":
        return Es * s2 / (Es + s2)
    raise ValueError(kind)


def fixed_point(kind: str, beta: float, N0: float, Es: float = 1.0, w: float = 1.0) -> float:
    """Decoupled noise variance: the largest root of ``w sigma^2 = N0 + beta Psi(sigma^2)``.

    ``w = 1`` is Thm. 1 (centralized / PD); ``w = w_c`` is Lemma 2 (one FD cluster).
    Solved by bisection on ``f(s) = w s - N0 - beta Psi(s)``, which is negative at
    ``s -> 0+`` (for N0 > 0) and positive for large ``s`` when a root exists.
    """
    if kind == "zf" and w <= beta:
        return math.inf
    f = lambda s: w * s - N0 - beta * psi(kind, s, Es)
    hi = 1.0
    while f(hi) <= 0.0:
        hi *= 2.0
        if hi > 1e300:
            return math.inf
    lo = 0.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return hi


def sinr_pd(kind: str, beta: float, snr: float) -> float:
    """Closed-form post-equalization SINR of Cor. 1 (``snr = Es/N0``)."""
    if kind == "mrc":
        return snr / (1.0 + beta * snr)
    if kind == "zf":
        if beta >= 1.0:
            raise ValueError("ZF needs beta < 1")
        return snr * (1.0 - beta)
    if kind == "lmmse":
        a = 1.0 - snr * (1.0 - beta)
        return 0.5 * (math.sqrt(a * a + 4.0 * snr) - a)
    raise ValueError(kind)


def sinr_fd_lmmse(beta: float, snr: float, w) -> float:
    """Post-fusion L-MMSE SINR for cluster fractions ``w`` (Lemma 5, Eq. LMMSE_equalization)."""
    w = np.asarray(w, dtype=np.float64)
    C = len(w)
    root = np.sqrt((1.0 - snr * (w - beta)) ** 2 + 4.0 * snr * w).sum()
    return float(0.5 * root - 0.5 * (C - snr * (1.0 - C * beta)))


def sinr_fd_lmmse_uniform(beta: float, snr: float, C: int) -> float:
    """Lower bound of Lemma 7, attained by uniform clusters ``w_c = 1/C``.

    Written as the proof of Lemma 7 derives it: Jensen's inequality on the
    convex summand ``f(w)`` of Lemma 5 gives ``sum_c f(w_c) >= C f(1/C)``, i.e.
    ``0.5 sqrt((C - x)^2 + 4 snr C) - 0.5 (C - x)`` with ``x = snr (1 - C beta)``.
    The displayed Eq. LMMSE_lower has ``1 - x`` inside the square; that form
    disagrees with Lemma 5 at ``w_c = 1/C`` whenever ``C > 1``, so the
    derivation's form is used.
    """
    x = snr * (1.0 - C * beta)
    return 0.5 * math.sqrt((C - x) ** 2 + 4.0 * snr * C) - 0.5 * (C - x)


def sinr_fd_zf(beta: float, snr: float, C: int) -> float:
    """Post-fusion ZF SINR ``(Es/N0)(1 - C beta)`` for ``w_c >= beta`` (Lemma 4)."""
    return snr * (1.0 - C * beta)


def message_entries(U: int, n_sc: int, n_sym: int, C: int) -> tuple[int, int]:
    """Complex entries sent to the fusion unit (Sec. VI-B): ``(m_PD, m_FD)``."""
    m_pd = U * U * n_sc * C + U * n_sc * n_sym * C
    m_fd = U * n_sc * n_sym * C
    return m_pd, m_fd
