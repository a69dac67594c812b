"""FP64 oracle: MRC and ZF equalization for the PD and FD architectures.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Written from the paper's definitions (Sec. III-A for PD; the FD architecture of
Sec. IV-A applies the same equalizer per cluster and fuses the local estimates
with the optimal weights of Lemma 1, Eq. fusionrule and opt_fusion, whose
variance is that of Thm. 3):

* MRC:  ``z = diag(G)^{-1} y^MRC`` with the error variance
  ``diag(diag(G)^{-1} G diag(G)^{-H} N0 + (diag(G)^{-1} G - I)(diag(G)^{-1} G - I)^H Es)``;
* ZF:   ``z = G^{-1} y^MRC`` with ``sigma^2 = N0 diag(G^{-1})``.

Both estimates are unbiased (the coefficient of ``s_u`` in ``z_u`` is 1), so the
fusion uses them as they are.  The fused variance is Thm. 3's
``(sum_c sigma_c^-2)^-1``; for ZF it is the exact MSE given ``H`` (the cluster
errors are noise on disjoint antennas), for MRC it is the paper's model value
(the clusters' interference terms share ``s``).  Readings (shared with the
kernels): a user a cluster cannot see (``G_uu = 0``) gets weight 0 (infinite
variance).  PD-MRC is ``z = diag(G)^{-1} y^MRC`` with its variance and no
fusion step.  A variance of exactly 0 happens only with ``N0 = 0``: for ZF
always, for MRC when the user has no interference in that cluster
(``G_uv = 0`` for every ``v != u``: a single user, or channels of disjoint
support).  The weights are then those of the limit ``N0 -> 0`` of Lemma 1's
weights ``sigma_c^-2 / sum sigma^-2``: ZF ``sigma_c^2 = N0 [G_c^{-1}]_uu``
gives weights proportional to ``1 / [G_c^{-1}]_uu``; MRC
``sigma_c^2 = (N0 G_uu + Es I_c) / G_uu^2`` (``I_c`` the interference sum) is
``~ N0 / G_uu`` where ``I_c = 0`` and stays positive elsewhere, so per user the
zero-interference clusters share all the weight in proportion to ``G_c,uu`` and
the fused variance is 0; a user with interference in every cluster keeps the
ordinary weights.  ZF needs ``G`` (FD: every ``G_c``) positive definite;
``info`` is the first non-positive leading minor as for L-MMSE (parity pinned
for clusters of at least ``U`` antennas).
"""
from __future__ import annotations

import numpy as np

from .lmmse import _as_math, first_nonpositive_minor, local_preprocess, optimal_fusion, partition

__all__ = ["mrc_unit", "mrc_fusion", "zf_unit", "equalize_pd_linear", "equalize_fd_linear"]


def mrc_unit(G: np.ndarray, yMR: np.ndarray, N0: float, Es: float):
    """MRC on ``(G, y^MRC)`` (Sec. III-A): ``(z, sigma2, g)`` with ``g = diag(G)``
    (what the ``N0 -> 0`` limit weights use)."""
    U = G.shape[0]
    g = np.real(np.diag(G))
    seen = g > 0
    Dinv = np.diag(np.where(seen, 1.0 / np.where(seen, g, 1.0), 0.0))
    z = Dinv @ yMR
    E = Dinv @ G - np.eye(U)
    np.fill_diagonal(E, 0.0)     # [diag(G)^{-1} G]_uu = 1 exactly; (1/g) g - 1 would leave rounding
    sigma2 = np.real(np.diag(Dinv @ G @ Dinv.conj().T * N0 + E @ E.conj().T * Es))
    sigma2 = np.where(seen, sigma2, np.inf)
    return z, sigma2, g


def mrc_fusion(z_c: np.ndarray, sigma2_c: np.ndarray, g_c: np.ndarray):
    """Lemma 1 fusion of MRC pairs ``z_c [C][U][n_sym]``, ``sigma2_c [C][U]``,
    ``g_c = G_c,uu [C][U]``, user by user: where some seen cluster has variance
    exactly 0 (``N0 = 0``, no interference there) the weights are the limit ones,
    ``g_c / sum g`` over those clusters, and the fused variance is 0; otherwise
    the ordinary optimal fusion (Eq. opt_fusion, Thm. 3)."""
    z, s2, nu = optimal_fusion(z_c, sigma2_c)
    zero = (g_c > 0) & (sigma2_c == 0.0)
    for u in np.nonzero(zero.any(axis=0))[0]:
        w = np.where(zero[:, u], g_c[:, u], 0.0)
        nu[:, u] = w / w.sum()
        z[u] = np.einsum("c,cn->n", nu[:, u], z_c[:, u])
        s2[u] = 0.0
    return z, s2, nu


def zf_unit(G: np.ndarray, yMR: np.ndarray, N0: float, Es: float):
    """ZF on ``(G, y^MRC)``: ``(z, sigma2, A, info)`` with ``A = G^{-1}``."""
    U = G.shape[0]
    info = first_nonpositive_minor(G)
    if info:
        nan = np.full(U, np.nan)
        return np.full(yMR.shape, np.nan + 0j), nan, np.full((U, U), np.nan + 0j), info
    A = np.linalg.inv(G)
    z = A @ yMR
    sigma2 = N0 * np.real(np.diag(A))
    return z, sigma2, A, 0


def _pd_gram(Hm, Ym, bounds):
    U, n_sym = Hm.shape[1], Ym.shape[1]
    G = np.zeros((U, U), np.complex128)
    yMR = np.zeros((U, n_sym), np.complex128)
    for b0, b1 in bounds:                         # the adder tree of Eq. fullMRC
        Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
        G += Gc
        yMR += yc
    return G, yMR


def equalize_pd_linear(H, y, N0: float, Es: float, C: int, equalizer: str, cluster_sizes=None) -> dict:
    """PD with MRC or ZF: ``z [n_sc][n_sym][U]``, ``sigma2 [n_sc][U]``, ``info [n_sc][1]``."""
    if equalizer not in ("mrc", "zf"):
        raise ValueError(equalizer)
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    s2 = np.zeros((n_sc, U))
    info = np.zeros((n_sc, 1), np.int32)
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        G, yMR = _pd_gram(Hm, Ym, bounds)
        if equalizer == "mrc":
            zk, s2k, _ = mrc_unit(G, yMR, N0, Es)   # the paper's z = diag(G)^{-1} y^MRC, no fusion
        else:
            zk, s2k, _, inf = zf_unit(G, yMR, N0, Es)
            info[k, 0] = inf
        z[k], s2[k] = zk.T, s2k
    return {"z": z, "sigma2": s2, "info": info}


def equalize_fd_linear(H, y, N0: float, Es: float, C: int, equalizer: str, cluster_sizes=None) -> dict:
    """FD with MRC or ZF per cluster and the optimal fusion (Lemma 1, Thm. 3)."""
    if equalizer not in ("mrc", "zf"):
        raise ValueError(equalizer)
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    s2 = np.zeros((n_sc, U))
    info = np.zeros((n_sc, C), np.int32)
    for k in range(n_sc):
        Hm, Ym = _as_math(H, y, k)
        zc = np.zeros((C, U, n_sym), np.complex128)
        s2c = np.zeros((C, U))
        gc = np.zeros((C, U))
        wvar = np.zeros((C, U))
        for c, (b0, b1) in enumerate(bounds):
            Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
            if equalizer == "mrc":
                zc[c], s2c[c], gc[c] = mrc_unit(Gc, yc, N0, Es)
            else:
                zc[c], s2c[c], A, info[k, c] = zf_unit(Gc, yc, N0, Es)
                if not info[k, c]:
                    wvar[c] = np.real(np.diag(A))
        if info[k].any():
            z[k], s2[k] = np.nan, np.nan
            continue
        if equalizer == "mrc":
            zf_, s2f, _ = mrc_fusion(zc, s2c, gc)
        else:
            # N0 = 0: every ZF variance vanishes; the weights of the limit N0 -> 0.
            zf_, s2f, _ = optimal_fusion(zc, s2c, weight_var=wvar if N0 == 0.0 else None)
        z[k], s2[k] = zf_.T, s2f
    return {"z": z, "sigma2": s2, "info": info}
