"""FP64 oracle: differentiable FD equalization and its adjoint.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper fixes the FD architecture (Sec. II-D, Sec. IV-A) with the L-MMSE
regularizer rho = N0/Es (Sec. III-A) and fusion weights from Lemma 1.  Its
trainable form -- per-cluster regularizers ``rho_c`` and explicit real fusion
weights ``nu[c][u]`` shared by all subcarriers, tuned on a loss -- is not in the
paper; reading taken here:

    x_c = (G_c + rho_c I)^{-1} H_c^H y_c          (local estimate, per symbol)
    z_u = sum_c nu[c][u] x_{c,u}                   (Eq. fusionrule with free weights)

Complex gradients follow the convention ``g = dL/dRe + i dL/dIm`` of a real loss
``L``.  With ``M_c = G_c + rho_c I`` (Hermitian), ``G_x,c = diag(nu_c) G_z`` and
``G_b,c = M_c^{-1} G_x,c`` (matrices over the n_sym right-hand sides):

    dL/dH_c   = Y_c G_b^H - H_c (G_b X_c^H + X_c G_b^H)      (B_c x U)
    dL/dy_c   = H_c G_b                                      (B_c x n_sym)
    dL/drho_c = -Re tr(G_b^H X_c)                           (summed over subcarriers)
    dL/dnu[c][u] = sum_n Re(conj(g_z,u,n) x_c,u,n)           (summed over subcarriers)

(from dX = M^{-1}(dB - dM X), dM = dH^H H + H^H dH + drho I, dB = dH^H Y + H^H dY).
``finite_difference`` checks them against the definition of the derivative.
"""
from __future__ import annotations

import numpy as np

from .lmmse import partition

__all__ = ["fd_train_forward", "fd_train_backward", "fd_optimal_backward", "finite_difference"]


def _blocks(H, y, k, bounds):
    Hm = np.asarray(H[k], dtype=np.complex128).T          # B x U
    Ym = np.asarray(y[k], dtype=np.complex128).T          # B x n_sym
    return [(Hm[b0:b1], Ym[b0:b1]) for (b0, b1) in bounds]


def fd_train_forward(H, y, rho, nu, cluster_sizes=None):
    """Return ``z`` ``[n_sc][n_sym][U]`` and the local estimates ``x`` ``[n_sc][C][n_sym][U]``.

    ``cluster_sizes``: the antennas of each cluster (Sec. II-B, contiguous, summing
    to B); ``None`` for C clusters of B / C."""
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    C = len(rho)
    bounds = partition(B, C, cluster_sizes)
    z = np.zeros((n_sc, n_sym, U), np.complex128)
    xs = np.zeros((n_sc, C, n_sym, U), np.complex128)
    for k in range(n_sc):
        for c, (Hc, Yc) in enumerate(_blocks(H, y, k, bounds)):
            M = Hc.conj().T @ Hc + rho[c] * np.eye(U)
            X = np.linalg.solve(M, Hc.conj().T @ Yc)             # U x n_sym
            xs[k, c] = X.T
            z[k] += (nu[c][:, None] * X).T
    return z, xs


def fd_train_backward(H, y, rho, nu, gz, cluster_sizes=None):
    """Gradients of a real loss with ``dL/dz = gz`` (``[n_sc][n_sym][U]``, dL/dRe + i dL/dIm).

    Returns ``(gH [n_sc][U][B], gy [n_sc][n_sym][B], grho [C], gnu [C][U])``;
    ``cluster_sizes`` as for ``fd_train_forward``.
    """
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    C = len(rho)
    bounds = partition(B, C, cluster_sizes)
    gH = np.zeros((n_sc, U, B), np.complex128)
    gy = np.zeros((n_sc, n_sym, B), np.complex128)
    grho = np.zeros(C)
    gnu = np.zeros((C, U))
    for k in range(n_sc):
        Gz = np.asarray(gz[k], dtype=np.complex128).T             # U x n_sym
        for c, (Hc, Yc) in enumerate(_blocks(H, y, k, bounds)):
            M = Hc.conj().T @ Hc + rho[c] * np.eye(U)
            X = np.linalg.solve(M, Hc.conj().T @ Yc)
            Gx = nu[c][:, None] * Gz
            Gb = np.linalg.solve(M, Gx)                           # M Hermitian: M^{-H} = M^{-1}
            b0, b1 = bounds[c]
            gH[k, :, b0:b1] = (Yc @ Gb.conj().T - Hc @ (Gb @ X.conj().T + X @ Gb.conj().T)).T
            gy[k, :, b0:b1] = (Hc @ Gb).T
            grho[c] += -np.real(np.trace(Gb.conj().T @ X))
            gnu[c] += np.real(np.sum(np.conj(Gz) * X, axis=1))
    return gH, gy, grho, gnu


def fd_optimal_backward(H, y, N0: float, Es: float, C: int, gz, cluster_sizes=None):
    """Gradients through the optimal-weight rule: the FD estimate with the unbiased
    per-cluster pairs fused by Lemma 1 (``lmmse.equalize_fd(..., "unbiased")``, the
    forward the library computes), differentiated with respect to ``H`` and ``y``.

    Per subcarrier and cluster, with ``M_c = G_c + rho I``, ``A_c = M_c^{-1}``,
    ``X_c = A_c H_c^H Y_c``, ``a_c = diag(A_c)``, ``w_c = 1 / a_c``: the fused estimate is
    ``z_u = sum_c w_{c,u} X_{c,u} / D_u`` with ``D_u = sum_c (w_{c,u} - rho)`` (weights
    ``mu / (N0 a)`` with ``mu = 1 - rho a``; ``N0`` cancels).  Its differential
    ``dz_u = (sum_c w_{c,u} dX_{c,u} + (X_{c,u} - z_u) dw_{c,u}) / D_u`` with
    ``dw = -da / a^2``, ``dX = A (dB - dM X)``, ``da_u = -[A dM A]_uu`` gives, for
    ``G_x = diag(w_c / D) G_z``, ``G_b = A_c G_x`` and
    ``q_u = -Re(sum_n conj(g_z,u,n) (X_{c,u,n} - z_{u,n})) / (D_u a_{c,u}^2)``:

        dL/dH_c = Y_c G_b^H - H_c (X_c G_b^H + G_b X_c^H + 2 A_c diag(q) A_c)
        dL/dy_c = H_c G_b

    (the free-weight adjoint above plus the term of the weights' dependence on
    ``a_c``).  ``gz`` is ``dL/dRe z + i dL/dIm z`` ``[n_sc][n_sym][U]``; users whose
    gain ``mu`` is not positive are outside the smooth region and not handled.
    Returns ``(gH [n_sc][U][B], gy [n_sc][n_sym][B])``.
    """
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    bounds = partition(B, C, cluster_sizes)
    rho = N0 / Es
    gH = np.zeros((n_sc, U, B), np.complex128)
    gy = np.zeros((n_sc, n_sym, B), np.complex128)
    for k in range(n_sc):
        Gz = np.asarray(gz[k], dtype=np.complex128).T              # U x n_sym
        blocks = _blocks(H, y, k, bounds)
        As, Xs, ws = [], [], []
        for Hc, Yc in blocks:
            A = np.linalg.inv(Hc.conj().T @ Hc + rho * np.eye(U))
            As.append(A)
            Xs.append(A @ (Hc.conj().T @ Yc))
            ws.append(1.0 / np.real(np.diag(A)))
        D = sum(w - rho for w in ws)                                # [U]
        z = sum(w[:, None] * X for w, X in zip(ws, Xs)) / D[:, None]
        for c, (Hc, Yc) in enumerate(blocks):
            A, X, w = As[c], Xs[c], ws[c]
            a = 1.0 / w
            Gb = A @ ((w / D)[:, None] * Gz)
            q = -np.real(np.sum(np.conj(Gz) * (X - z), axis=1)) / (D * a * a)
            K = X @ Gb.conj().T + Gb @ X.conj().T + 2.0 * A @ np.diag(q) @ A
            b0, b1 = bounds[c]
            gH[k, :, b0:b1] = (Yc @ Gb.conj().T - Hc @ K).T
            gy[k, :, b0:b1] = (Hc @ Gb).T
    return gH, gy


def finite_difference(f, x: np.ndarray, eps: float = 1e-6) -> np.ndarray:
    """Central differences of the real scalar ``f`` at ``x``: ``dL/dRe + i dL/dIm`` for complex ``x``."""
    x = np.array(x, dtype=np.complex128 if np.iscomplexobj(x) else np.float64)
    g = np.zeros_like(x)
    flat = x.reshape(-1)
    gf = g.reshape(-1)
    for i in range(flat.size):
        for unit in ((1.0, 1j) if np.iscomplexobj(x) else (1.0,)):
            old = flat[i]
            flat[i] = old + eps * unit
            fp = f(x)
            flat[i] = old - eps * unit
            fm = f(x)
            flat[i] = old
            gf[i] += unit * (fp - fm) / (2 * eps)
    return g
