"""FP64 oracle: max-log bit LLRs for square QAM.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper says that the equalizer output ``{z, sigma^2}`` feeds a soft-output
detector that computes log-likelihood ratios (Sec. II-A, Sec. III-A) but gives
no formula.  Reading taken here, applied to the decoupled scalar channel
``z_u = s_u + e_u`` with ``e_u ~ CN(0, sigma_u^2)`` (Eq. 4):

* Alphabet: ``L x L`` square QAM, ``L = 2^(bits/2)``, odd-integer levels
  ``2i - (L-1)`` per axis, scaled to average energy ``Es``.
* Labels: the first ``bits/2`` bits are the binary-reflected Gray code of the
  in-phase level index ``i`` (``i ^ (i >> 1)``, most significant bit first), the
  last ``bits/2`` bits the same for the quadrature index.
* LLR of bit ``b``: ``(min_{a: b(a)=1} |z-a|^2 - min_{a: b(a)=0} |z-a|^2) / sigma^2``
  (max-log; positive favours bit 0).  ``sigma^2 = inf`` gives 0; ``sigma^2 = 0``
  gives +-inf (0 on an exact tie).

The oracle enumerates all ``L^2`` points of the two-dimensional alphabet.
"""
from __future__ import annotations

import numpy as np

__all__ = ["qam_alphabet", "maxlog_llr", "hard_bits"]


def qam_alphabet(bits: int, Es: float = 1.0):
    """Return ``(points [M] complex128, labels [M][bits] int)`` of the labelled QAM alphabet."""
    if bits not in (2, 4, 6, 8):
        raise ValueError("bits must be 2, 4, 6 or 8")
    L = 1 << (bits // 2)
    h = bits // 2
    scale = np.sqrt(Es / (2.0 * (L * L - 1) / 3.0))
    pts, labels = [], []
    for iI in range(L):
        for iQ in range(L):
            pts.append(((2 * iI - (L - 1)) + 1j * (2 * iQ - (L - 1))) * scale)
            gI, gQ = iI ^ (iI >> 1), iQ ^ (iQ >> 1)
            lab = [(gI >> (h - 1 - t)) & 1 for t in range(h)] + [(gQ >> (h - 1 - t)) & 1 for t in range(h)]
            labels.append(lab)
    return np.array(pts), np.array(labels, dtype=np.int64)


def maxlog_llr(z: np.ndarray, sigma2: np.ndarray, bits: int, Es: float = 1.0) -> np.ndarray:
    """Max-log LLRs.  ``z`` ``[..., U]`` complex, ``sigma2`` broadcastable to ``z``; returns ``[..., U, bits]``."""
    pts, labels = qam_alphabet(bits, Es)
    z = np.asarray(z, dtype=np.complex128)
    d = np.abs(z[..., None] - pts) ** 2                        # [..., U, M]
    out = np.empty(z.shape + (bits,))
    s2 = np.broadcast_to(np.asarray(sigma2, dtype=np.float64), z.shape)
    for b in range(bits):
        d1 = np.min(np.where(labels[:, b] == 1, d, np.inf), axis=-1)
        d0 = np.min(np.where(labels[:, b] == 0, d, np.inf), axis=-1)
        diff = d1 - d0
        with np.errstate(divide="ignore", invalid="ignore"):
            v = diff / s2
        v = np.where(np.isinf(s2), 0.0, v)
        v = np.where((s2 == 0) & (diff == 0), 0.0, v)
        out[..., b] = v
    return out


def hard_bits(levels: np.ndarray, bits: int) -> np.ndarray:
    """Labels of transmitted points from per-axis level indices ``[..., 2]`` -> ``[..., bits]``."""
    h = bits // 2
    lv = np.asarray(levels, dtype=np.int64)
    g = lv ^ (lv >> 1)
    out = np.empty(lv.shape[:-1] + (bits,), dtype=np.int64)
    for t in range(h):
        out[..., t] = (g[..., 0] >> (h - 1 - t)) & 1
        out[..., h + t] = (g[..., 1] >> (h - 1 - t)) & 1
    return out
