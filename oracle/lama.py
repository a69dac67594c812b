"""FP64 oracle: LAMA equalization for the PD and FD architectures.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

LAMA-PD (Sec. III-B, Algorithm 1, Eq. LAMA_Gaussian and Eq. F) iterates on the
PD pair ``(G, y^MRC)``; the error variance of ``z^t`` is ``N0 + beta phi^t``.
LAMA-FD runs the same algorithm on each cluster's ``(G_c, y_c^MRC)`` and fuses
the per-cluster estimates with the optimal weights of Lemma 1 (Thm. 3,
Lemma 5 for the per-cluster variances).

Readings (shared with the kernels):

* **Normalization.**  Algorithm 1 is written for the paper's Rayleigh model,
  entries of ``H`` of variance ``1/B`` (so ``G ~ I``).  With the inputs' CN(0, 1)
  entries it runs on ``G / B``, ``y^MRC / B`` and ``N0 / B`` with
  ``beta = U / B``.  A cluster of ``S_c`` antennas is the system
  ``H_c / sqrt(S_c)`` of ratio ``beta_c = U / S_c`` and noise ``N0 / S_c``: the
  per-cluster fixed point of Lemma 5, ``w_c sigma_c^2 = N0 + beta Psi(sigma_c^2)``,
  written in that cluster's own units.
* **Prior** (Eq. prior): equiprobable square QAM, the constellation of the LLRs
  (odd-integer levels scaled to ``Es``).  ``F`` and ``G`` are the posterior mean
  and variance of Eq. F under ``z = s + CN(0, tau)``, here by brute force over
  every constellation point.
* **Iterations.**  ``T`` iterations compute ``z^1..z^T`` (and ``T - 1`` denoiser
  steps between them); the output is ``z^T`` with ``sigma^2 = N0 + beta phi^T``,
  the variance Algorithm 1 attaches to ``z^T``.  ``T = 1`` gives the normalized
  matched filter with ``sigma_1^2 = N0 + beta Es`` (the initial value of Thm. 2).
  ``<.>`` (Sec. II-A) averages over the ``U`` users.
* **Per receive vector.**  ``phi^t`` depends on the received vector, so the
  variance is per (subcarrier, symbol), shared by the users: ``sigma2`` is
  ``[n_sc][n_sym][U]``.
* **FD fusion.**  The per-cluster variance is the same for every user, so the
  weights are ``(1/sigma_c^2) / sum_c' (1/sigma_c'^2)``; an empty cluster has
  weight 0.  ``N0 > 0`` is required (the denoiser needs ``tau > 0``).
"""
from __future__ import annotations

import numpy as np

from .lmmse import _as_math, local_preprocess, partition

__all__ = ["qam_points", "denoise", "lama_unit", "equalize_pd_lama", "equalize_fd_lama"]


def qam_points(bits: int, Es: float) -> np.ndarray:
    """The ``2^bits`` points of square QAM: odd-integer levels per axis scaled to energy ``Es``."""
    L = 1 << (bits // 2)
    lev = np.arange(-(L - 1), L, 2, dtype=np.float64)
    e_avg = 2.0 * np.mean(lev ** 2)
    lev = lev * np.sqrt(Es / e_avg)
    return (lev[:, None] + 1j * lev[None, :]).ravel()


def denoise(z: np.ndarray, tau: float, points: np.ndarray):
    """Posterior mean ``F(z, tau)`` and variance ``G(z, tau)`` of Eq. F, element-wise:
    ``p(s | z) ~ exp(-|z - s|^2 / tau)`` over the equiprobable ``points``."""
    zf = np.asarray(z).reshape(-1)
    e = -np.abs(zf[:, None] - points[None, :]) ** 2 / tau
    e -= e.max(axis=1, keepdims=True)
    w = np.exp(e)
    w /= w.sum(axis=1, keepdims=True)
    F = w @ points
    G = w @ np.abs(points) ** 2 - np.abs(F) ** 2
    return F.reshape(np.shape(z)), np.maximum(G, 0.0).reshape(np.shape(z))


def lama_unit(G: np.ndarray, yMR: np.ndarray, N0: float, Es: float, beta: float, points, T: int):
    """Algorithm 1 on a normalized pair (``G ~ I``) for each column of ``yMR`` (``U x n_sym``).

    Returns ``(z^T [U][n_sym], sigma2 [n_sym])`` with ``sigma2 = N0 + beta phi^T``.
    """
    U, n_sym = yMR.shape
    z_out = np.zeros((U, n_sym), np.complex128)
    s2_out = np.zeros(n_sym)
    IG = np.eye(U) - G
    for n in range(n_sym):
        s = np.zeros(U, np.complex128)                # E[S] = 0 (zero-mean constellation)
        phi = Es                                      # Var[S]
        v = np.zeros(U, np.complex128)
        for t in range(1, T + 1):
            z = yMR[:, n] + IG @ s + v
            tau = N0 + beta * phi
            if t == T:
                break
            s_new, g = denoise(z, tau, points)
            phi_new = float(np.mean(g))
            v = beta * phi_new / tau * (z - s)
            s, phi = s_new, phi_new
        z_out[:, n] = z
        s2_out[n] = tau
    return z_out, s2_out


def equalize_pd_lama(H, y, N0: float, Es: float, C: int, bits: int, T: int, cluster_sizes=None) -> dict:
    """LAMA-PD: ``z [n_sc][n_sym][U]``, ``sigma2 [n_sc][n_sym][U]``."""
    if not N0 > 0:
        raise ValueError("LAMA needs N0 > 0")
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    pts = qam_points(bits, Es)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    s2 = np.zeros((n_sc, n_sym, U))
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        G = np.zeros((U, U), np.complex128)
        yMR = np.zeros((U, n_sym), np.complex128)
        for b0, b1 in bounds:                         # Eq. fullMRC
            Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
            G += Gc
            yMR += yc
        zk, s2k = lama_unit(G / B, yMR / B, N0 / B, Es, U / B, pts, T)
        z[k] = zk.T
        s2[k] = s2k[:, None]
    return {"z": z, "sigma2": s2}


def equalize_fd_lama(H, y, N0: float, Es: float, C: int, bits: int, T: int, cluster_sizes=None) -> dict:
    """LAMA-FD: LAMA per cluster, then the optimal fusion (Lemma 1, Thm. 3)."""
    if not N0 > 0:
        raise ValueError("LAMA needs N0 > 0")
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    pts = qam_points(bits, Es)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    s2 = np.zeros((n_sc, n_sym, U))
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        num = np.zeros((U, n_sym), np.complex128)
        den = np.zeros(n_sym)
        for b0, b1 in bounds:
            S = b1 - b0
            if S == 0:
                continue                              # sees no user: weight 0
            Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
            zc, s2c = lama_unit(Gc / S, yc / S, N0 / S, Es, U / S, pts, T)
            num += zc / s2c[None, :]
            den += 1.0 / s2c
        z[k] = (num / den[None, :]).T
        s2[k] = (1.0 / den)[:, None]
    return {"z": z, "sigma2": s2}
