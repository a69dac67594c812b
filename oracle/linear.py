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
(the clusters' interference terms share ``s``).  Readings (shared with the kernels): a user a
cluster cannot see (``G_uu = 0``) gets weight 0 (infinite variance); for
``N0 = 0`` every ZF variance is 0 and the fusion weights are taken in the limit
``N0 -> 0`` (proportional to ``1 / [G_c^{-1}]_uu``); MRC variances with
``N0 = 0`` are zero only without interference (``U = 1``), then the weights are
proportional to ``G_uu``.  Outside that limit a variance of exactly 0 (``N0 = 0``
and a user with no interference in that cluster, a set of channels of measure
zero) leaves the weight ``1 / sigma^2`` undefined: such a pair gets weight 0,
in PD (one pair through the same rule) as in FD.  ZF needs ``G`` (FD: every ``G_c``) positive definite;
``info`` is the first non-positive leading minor as for L-MMSE (parity pinned
for clusters of at least ``U`` antennas).
"""
from __future__ import annotations

import numpy as np

from .lmmse import _as_math, first_nonpositive_minor, local_preprocess, optimal_fusion, partition

__all__ = ["mrc_unit", "zf_unit", "equalize_pd_linear", "equalize_fd_linear"]


def mrc_unit(G: np.ndarray, yMR: np.ndarray, N0: float, Es: float):
    """MRC on ``(G, y^MRC)``: ``(z, sigma2, weight_var)``; ``weight_var`` is what
    the fusion weights use when ``sigma2`` vanishes (``N0 = 0``, no interference)."""
    U = G.shape[0]
    g = np.real(np.diag(G))
    seen = g > 0
    Dinv = np.diag(np.where(seen, 1.0 / np.where(seen, g, 1.0), 0.0))
    z = Dinv @ yMR
    E = Dinv @ G - np.eye(U)
    np.fill_diagonal(E, 0.0)     # [diag(G)^{-1} G]_uu = 1 exactly; (1/g) g - 1 would leave rounding
    sigma2 = np.real(np.diag(Dinv @ G @ Dinv.conj().T * N0 + E @ E.conj().T * Es))
    sigma2 = np.where(seen, sigma2, np.inf)
    weight_var = np.where(seen, 1.0 / np.where(seen, g, 1.0), np.inf)
    return z, sigma2, weight_var


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
            # One estimate passed through the fusion rule, so that PD and FD at
            # C = 1 agree in the degenerate cases too (a variance of exactly 0
            # outside the N0 -> 0 limit carries no weight).
            zk, s2k, wv = mrc_unit(G, yMR, N0, Es)
            limit = N0 == 0.0 and U == 1
            zk, s2k, _ = optimal_fusion(zk[None], s2k[None], weight_var=wv[None] if limit else None)
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
        wvar = np.zeros((C, U))
        for c, (b0, b1) in enumerate(bounds):
            Gc, yc = local_preprocess(Hm[b0:b1], Ym[b0:b1])
            if equalizer == "mrc":
                zc[c], s2c[c], wvar[c] = mrc_unit(Gc, yc, N0, Es)
            else:
                zc[c], s2c[c], A, info[k, c] = zf_unit(Gc, yc, N0, Es)
                if not info[k, c]:
                    wvar[c] = np.real(np.diag(A))
        if info[k].any():
            z[k], s2[k] = np.nan, np.nan
            continue
        # Vanishing variances (N0 = 0: ZF always, MRC without interference): the
        # weights of the limit N0 -> 0.
        limit = N0 == 0.0 and (equalizer == "zf" or U == 1)
        zf_, s2f, _ = optimal_fusion(zc, s2c, weight_var=wvar if limit else None)
        z[k], s2[k] = zf_.T, s2f
    return {"z": z, "sigma2": s2, "info": info}
