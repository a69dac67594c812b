"""FP64 oracle: PD and FD L-MMSE equalization with optimal fusion.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Data layout (shared with the generator, not with the CUDA path):
``H[k]`` is ``[U][B]`` (the transpose of the paper's ``B x U`` matrix), ``y[k]``
is ``[n_sym][B]``.  Inside each function the paper's matrices are formed
explicitly: ``Hm = H[k].T`` (``B x U``), ``Ym = y[k].T`` (``B x n_sym``).

Readings of the paper taken here (the paper is silent or ambiguous on them):

* Error variance ``sigma^2`` is real (the paper types it complex in Sec. II-C).
* ``estimate='literal'`` returns the paper's L-MMSE estimate
  ``z = (G + rho I)^{-1} y^MRC`` and its error variance from the formula of
  Sec. III-A.  ``estimate='unbiased'`` divides by the per-user gain
  ``mu_u = [(G + rho I)^{-1} G]_uu`` so that ``z_u = s_u + e_u`` holds as in the
  decoupled model (Eq. 4) that Lemma 1's proof assumes; its error variance is
  the variance of that unbiased error, ``(sigma^2 - (1 - mu)^2 Es) / mu^2``.
* FD fusion (Eq. fusionrule, Lemma 1) fuses the per-cluster pairs of the chosen
  kind; the fused variance is ``(sum_c sigma_c^-2)^-1`` (Thm. 3, Eq. sigma_FD).
* ``N0 = 0`` (zero forcing, ``rho = 0``): every error variance is zero and the
  weights of Eq. opt_fusion are taken in the limit ``N0 -> 0``, where they are
  proportional to ``mu_c / [A_c]_uu`` (unbiased) or ``1 / [A_c]_uu`` (literal).
* A user whose gain is ``mu <= 0`` (e.g. an all-zero channel column) has an
  infinite unbiased error variance, weight zero and estimate zero.
* ``info`` reports, per system matrix, the first ``k`` (1-based) whose leading
  ``k x k`` principal minor of ``G + rho I`` is not positive (0 if positive
  definite).  Outputs of such instances are NaN.
"""
from __future__ import annotations

import numpy as np

__all__ = ["partition", "local_preprocess", "lmmse_unit", "unbias", "optimal_fusion",
           "first_nonpositive_minor", "equalize_pd", "equalize_fd", "centralized_lmmse"]


def partition(B: int, C: int, cluster_sizes=None) -> list[tuple[int, int]]:
    """Contiguous antenna clusters ``B_c = w_c B`` (Sec. II-B).  Uniform when sizes are omitted."""
    if cluster_sizes is None:
        if C <= 0 or B % C:
            raise ValueError("uniform partition needs C > 0 dividing B")
        cluster_sizes = [B // C] * C
    if len(cluster_sizes) != C or sum(cluster_sizes) != B or min(cluster_sizes) < 0:
        raise ValueError("cluster sizes must be C non-negative integers summing to B")
    bounds, start = [], 0
    for bc in cluster_sizes:
        bounds.append((start, start + bc))
        start += bc
    return bounds


def local_preprocess(Hm_c: np.ndarray, Ym_c: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Local Gram matrix ``G_c = H_c^H H_c`` and MRC output ``y_c^MRC = H_c^H y_c`` (Sec. II-C)."""
    HhC = Hm_c.conj().T
    return HhC @ Hm_c, HhC @ Ym_c


def first_nonpositive_minor(M: np.ndarray) -> int:
    """First ``k`` (1-based) whose leading principal minor of Hermitian ``M`` is <= 0, else 0.

    ``M`` is positive definite iff all leading principal minors are positive
    (Sylvester's criterion); a Cholesky factorization stops at that ``k``.
    """
    for k in range(1, M.shape[0] + 1):
        if not np.real(np.linalg.det(M[:k, :k])) > 0.0:
            return k
    return 0


def lmmse_unit(G: np.ndarray, yMR: np.ndarray, N0: float, Es: float):
    """L-MMSE equalization on ``(G, y^MRC)`` (Sec. III-A).

    Returns ``(z, sigma2, A, mu, info)`` with ``A = (G + rho I)^{-1}``,
    ``rho = N0/Es``, the biased estimate ``z = A y^MRC`` (``U x n_sym``), the
    error variance from the paper's formula
    ``diag(A G A^H N0 + (A G - I)(A G - I)^H Es)`` and the gain ``mu = diag(A G)``.
    """
    U = G.shape[0]
    rho = N0 / Es
    M = G + rho * np.eye(U)
    info = first_nonpositive_minor(M)
    if info:
        nan = np.full(U, np.nan)
        return np.full(yMR.shape, np.nan + 0j), nan, np.full((U, U), np.nan + 0j), nan, info
    A = np.linalg.inv(M)
    z = A @ yMR
    AG = A @ G
    E = AG - np.eye(U)
    sigma2 = np.real(np.diag(A @ G @ A.conj().T * N0 + E @ E.conj().T * Es))
    mu = np.real(np.diag(AG))
    return z, sigma2, A, mu, 0


def unbias(z: np.ndarray, sigma2: np.ndarray, mu: np.ndarray, Es: float):
    """Unbiased estimate ``z/mu`` and the variance of its error ``(sigma2 - (1-mu)^2 Es)/mu^2``."""
    zu = np.zeros_like(z)
    s2u = np.full_like(sigma2, np.inf)
    ok = mu > 0
    zu[ok] = z[ok] / mu[ok, None]
    s2u[ok] = (sigma2[ok] - (1.0 - mu[ok]) ** 2 * Es) / mu[ok] ** 2
    return zu, s2u


def optimal_fusion(z_c: np.ndarray, sigma2_c: np.ndarray, weight_var=None):
    """Optimal linear fusion of per-cluster estimates (Eq. fusionrule, Lemma 1, Thm. 3).

    ``z_c``: ``[C][U][n_sym]``; ``sigma2_c``: ``[C][U]`` error variances.
    ``weight_var`` (same shape as ``sigma2_c``) replaces ``sigma2_c`` inside the
    weights only (used for the ``N0 -> 0`` limit).  Returns ``(z, sigma2, nu)``.
    """
    wv = sigma2_c if weight_var is None else weight_var
    inv = np.zeros_like(wv)
    good = np.isfinite(wv) & (wv > 0)
    inv[good] = 1.0 / wv[good]
    tot = inv.sum(axis=0)                                   # [U]
    nu = np.zeros_like(inv)
    has = tot > 0
    nu[:, has] = inv[:, has] / tot[has]                     # Eq. opt_fusion
    z = np.einsum("cu,cun->un", nu, z_c)                    # Eq. fusionrule
    sinv = np.zeros_like(tot)
    sg = np.isfinite(sigma2_c) & (sigma2_c > 0)
    sinv = np.where(sg, 1.0 / np.where(sg, sigma2_c, 1.0), 0.0).sum(axis=0)
    with np.errstate(divide="ignore"):
        sigma2 = np.where(sinv > 0, 1.0 / np.where(sinv > 0, sinv, 1.0), np.inf)  # Thm. 3
    if weight_var is not None:                              # N0 = 0: all variances are zero
        sigma2 = np.where(has, 0.0, np.inf)
    return z, sigma2, nu


def _as_math(H, y, k):
    Hm = np.asarray(H[k], dtype=np.complex128).T           # B x U
    Ym = np.asarray(y[k], dtype=np.complex128).T           # B x n_sym
    return Hm, Ym


def equalize_pd(H, y, N0: float, Es: float, C: int, estimate: str = "unbiased",
                cluster_sizes=None) -> dict:
    """PD architecture (Sec. II-C, Sec. III-A): local ``(G_c, y_c^MRC)``, adder tree, central L-MMSE.

    Returns ``z`` ``[n_sc][n_sym][U]``, ``sigma2`` ``[n_sc][U]``, ``mu``, ``info`` ``[n_sc]``.
    """
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    s2 = np.zeros((n_sc, U))
    mu_o = np.zeros((n_sc, U))
    info = np.zeros(n_sc, np.int32)
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        G = np.zeros((U, U), np.complex128)
        yMR = np.zeros((U, n_sym), np.complex128)
        for (b0, b1) in bounds:                               # Eq. fullMRC adder tree
            Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
            G += Gc
            yMR += yc
        zk, s2k, _, mu, inf = lmmse_unit(G, yMR, N0, Es)
        if estimate == "unbiased" and not inf:
            zk, s2k = unbias(zk, s2k, mu, Es)
        elif estimate not in ("unbiased", "literal"):
            raise ValueError(estimate)
        z[k] = zk.T
        s2[k] = s2k
        mu_o[k] = mu
        info[k] = inf
    return {"z": z, "sigma2": s2, "mu": mu_o, "info": info}


def equalize_fd(H, y, N0: float, Es: float, C: int, estimate: str = "unbiased",
                cluster_sizes=None) -> dict:
    """FD architecture (Sec. II-D, Sec. IV-A): local L-MMSE per cluster, then optimal fusion.

    Returns ``z`` ``[n_sc][n_sym][U]``, ``sigma2`` ``[n_sc][U]``, ``nu`` ``[n_sc][C][U]``,
    per-cluster ``z_c``/``sigma2_c`` and ``info`` ``[n_sc][C]``.
    """
    if estimate not in ("unbiased", "literal"):
        raise ValueError(estimate)
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    s2 = np.zeros((n_sc, U))
    nu_o = np.zeros((n_sc, C, U))
    zc_o = np.zeros((n_sc, C, n_sym, U), np.complex128)
    s2c_o = np.zeros((n_sc, C, U))
    info = np.zeros((n_sc, C), np.int32)
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        zc = np.zeros((C, U, n_sym), np.complex128)
        s2c = np.zeros((C, U))
        wvar = np.zeros((C, U))
        for c, (b0, b1) in enumerate(bounds):
            Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
            zk, s2k, A, mu, inf = lmmse_unit(Gc, yc, N0, Es)
            info[k, c] = inf
            if estimate == "unbiased" and not inf:
                zk, s2k = unbias(zk, s2k, mu, Es)
                with np.errstate(divide="ignore"):
                    wvar[c] = np.where(mu > 0, np.real(np.diag(A)) / np.where(mu > 0, mu, 1.0), np.inf)
            elif not inf:
                wvar[c] = np.real(np.diag(A))
            zc[c], s2c[c] = zk, s2k
        if info[k].any():
            z[k], s2[k] = np.nan, np.nan
            continue
        zf, s2f, nu = optimal_fusion(zc, s2c, weight_var=wvar if N0 == 0.0 else None)
        z[k] = zf.T
        s2[k] = s2f
        nu_o[k] = nu
        zc_o[k] = np.transpose(zc, (0, 2, 1))
        s2c_o[k] = s2c
    return {"z": z, "sigma2": s2, "nu": nu_o, "z_c": zc_o, "sigma2_c": s2c_o, "info": info}


def centralized_lmmse(H, y, N0: float, Es: float) -> np.ndarray:
    """Centralized L-MMSE as regularized least squares, solved by ``numpy.linalg.lstsq``.

    ``z = argmin_x ||y - H x||^2 + rho ||x||^2`` (the L-MMSE estimate of Sec. III-A),
    computed from the stacked system ``[H; sqrt(rho) I] x = [y; 0]`` with an
    SVD-based solver, i.e. without forming ``G`` or ``y^MRC``.  Used to pin
    ``equalize_pd`` by a different algorithm.
    """
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    rho = N0 / Es
    out = np.zeros((n_sc, n_sym, U), np.complex128)
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        Ab = np.vstack([Hm, np.sqrt(rho) * np.eye(U)])
        rhs = np.vstack([Ym, np.zeros((U, n_sym))])
        out[k] = np.linalg.lstsq(Ab, rhs, rcond=None)[0].T
    return out
