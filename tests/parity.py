"""Comparison helpers shared by the GPU parity tests (test infrastructure).

Two checks per subcarrier (the leading axis of every output array):

* norm:    ||x - x_oracle||_2 / ||x_oracle||_2 over all entries of the subcarrier;
* entries: |x - x_oracle| <= tol * max(|x_oracle|, rms(x_oracle)) for EVERY entry,
           rms taken over the subcarrier's entries, so one weak user's estimate
           cannot hide inside the norm of the others while entries near zero
           (an LLR at a decision threshold) are held to the subcarrier's scale.

``tol`` is a scalar or one bound per subcarrier.  Non-finite oracle entries
(sigma^2 = inf for a user no cluster sees, NaN for a failed factorization) must
be matched exactly by the GPU and are left out of both measures.
"""
from __future__ import annotations

import numpy as np


def _flat(a):
    a = np.asarray(a)
    return a.reshape(a.shape[0], -1) if a.ndim > 1 else a.reshape(-1, 1)


def rel_per_sc(a, b) -> np.ndarray:
    """||a - b|| / ||b|| per subcarrier over the finite entries of b."""
    a, b = _flat(a).astype(np.complex128), _flat(b).astype(np.complex128)
    fin = np.isfinite(b)
    d = np.where(fin, a - b, 0)
    bb = np.where(fin, b, 0)
    return np.linalg.norm(d, axis=1) / np.maximum(np.linalg.norm(bb, axis=1), 1e-30)


def entry_ratio(a, b) -> np.ndarray:
    """max over entries of |a - b| / max(|b|, rms(b)) per subcarrier (finite entries of b)."""
    a, b = _flat(a).astype(np.complex128), _flat(b).astype(np.complex128)
    fin = np.isfinite(b)
    bb = np.where(fin, b, 0)
    cnt = np.maximum(fin.sum(axis=1, keepdims=True), 1)
    rms = np.sqrt((np.abs(bb) ** 2).sum(axis=1, keepdims=True) / cnt)
    scale = np.maximum(np.abs(bb), np.maximum(rms, 1e-30))
    r = np.where(fin, np.abs(np.where(fin, a - b, 0)) / scale, 0.0)
    return r.max(axis=1)


def nonfinite_match(a, b) -> bool:
    """Where b is +-inf the GPU gives the same inf; where b is NaN the GPU gives NaN."""
    a, b = np.asarray(a), np.asarray(b)
    inf = np.isinf(b)
    nan = np.isnan(b)
    return bool(np.array_equal(a[inf], b[inf].astype(a.dtype)) and np.isnan(a[nan]).all())


def check(name: str, a, b, tol) -> tuple[float, float]:
    """Assert both measures within ``tol`` (scalar or per subcarrier); returns the worst
    (norm, entry) ratios for reporting."""
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, (name, a.shape, b.shape)
    assert nonfinite_match(a, b), f"{name}: non-finite entries differ from the oracle"
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), (a.shape[0],))
    en = rel_per_sc(a, b)
    ee = entry_ratio(a, b)
    k = int(np.argmax(en / tol))
    assert (en <= tol).all(), f"{name}: norm rel err {en[k]:.3g} > {tol[k]:.3g} (subcarrier {k})"
    k = int(np.argmax(ee / tol))
    assert (ee <= tol).all(), f"{name}: entry-wise rel err {ee[k]:.3g} > {tol[k]:.3g} (subcarrier {k})"
    return float(en.max()), float(ee.max())
