"""Seeded synthetic uplink data for the massive MU-MIMO system model.

This module is the data source of the system model (Sec. II-A, Eq. 1:
``y = H s0 + n``) and nothing else: it draws channels, transmit symbols and
noise, and forms the receive vectors.  It holds none of the equalizer's
arithmetic (no Gram matrix, no matched filter, no solve, no fusion, no LLR),
so both the FP64 oracle and the CUDA path can consume its output.

Conventions
-----------
* ``H`` has shape ``[n_sc][U][B]`` complex64: for subcarrier ``k`` the paper's
  ``B x U`` channel matrix stored user-major (``H[k][u][b]`` is the gain from
  user ``u`` to antenna ``b``; the antennas of one user are contiguous, which is
  the column-major layout of the paper's ``B x U`` matrix).
* ``y`` has shape ``[n_sc][n_sym][B]`` complex64 (one receive vector per OFDM
  symbol; the channel is constant over the ``n_sym`` symbols of a subcarrier).
* Channel entries are i.i.d. CN(0, 1).  The paper's Rayleigh model (Def. 2)
  uses CN(0, 1/B); scaling ``y`` by ``1/sqrt(B)`` maps one onto the other with
  ``N0_paper = N0 / B``.  The SNR is the paper's ``beta * Es / N0_paper``
  (Sec. V-A), which with CN(0, 1) entries is ``U * Es / N0``; hence
  ``N0 = U * Es / 10**(snr_db / 10)``.
* Optional receive-side exponential correlation ``R_ij = r**|i-j|`` over the
  whole array: ``H = R^{1/2} H_w`` with the Cholesky factor of ``R``.
* Transmit symbols are drawn uniformly (Eq. 2) from a square QAM alphabet with
  odd-integer levels ``{-(L-1), ..., -1, 1, ..., L-1}`` per axis, scaled to
  average energy ``Es``.  Only the level indices are drawn here; bit labels
  belong to the detector and are not defined in this module.

Random streams: one ``numpy`` PCG64 ``SeedSequence`` per call, spawned into
independent streams for H, symbols and noise, so that changing ``n_sym`` does
not change ``H`` and so on.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["Problem", "make_problem", "make_uneven", "noise_variance", "qam_levels", "exp_correlation"]


@dataclasses.dataclass
class Problem:
    """One seeded synthetic workload (all arrays on the host)."""

    H: np.ndarray          # complex64 [n_sc][U][B]
    y: np.ndarray          # complex64 [n_sc][n_sym][B]
    s: np.ndarray          # complex128 [n_sc][n_sym][U] transmitted symbols
    levels: np.ndarray     # int8 [n_sc][n_sym][U][2] per-axis level index (I, Q)
    N0: float
    Es: float
    B: int
    U: int
    C: int
    n_sc: int
    n_sym: int
    bits: int
    snr_db: float


def noise_variance(U: int, Es: float, snr_db: float) -> float:
    """Per-antenna noise variance giving the paper's SNR ``beta*Es/N0`` with CN(0,1) channels."""
    return float(U * Es / 10.0 ** (snr_db / 10.0))


def qam_levels(bits: int) -> tuple[int, float]:
    """Return ``(L, e_avg)``: levels per axis and average energy of the odd-integer grid."""
    if bits not in (2, 4, 6, 8):
        raise ValueError("bits per symbol must be 2, 4, 6 or 8")
    L = 1 << (bits // 2)
    e_avg = 2.0 * (L * L - 1) / 3.0
    return L, e_avg


def exp_correlation(B: int, r: float) -> np.ndarray:
    """Exponential correlation matrix ``R_ij = r**|i-j|`` (float64, B x B)."""
    idx = np.arange(B)
    return r ** np.abs(idx[:, None] - idx[None, :])


def make_problem(B: int, U: int, C: int, n_sc: int, n_sym: int, *, snr_db: float = 10.0,
                 bits: int = 4, seed: int = 0, Es: float = 1.0, corr_r: float | None = None,
                 noiseless: bool = False) -> Problem:
    """Draw one seeded workload of the uplink model ``y = H s0 + n``.

    ``C`` is carried along for bookkeeping (the data do not depend on it).
    ``noiseless=True`` sets ``n = 0`` and ``N0 = 0``.
    """
    if B <= 0 or U <= 0 or C <= 0 or n_sc < 0 or n_sym <= 0:
        raise ValueError("sizes must be positive (n_sc may be zero)")
    ss = np.random.SeedSequence(seed)
    g_h, g_s, g_n = (np.random.Generator(np.random.PCG64(c)) for c in ss.spawn(3))

    H = (g_h.standard_normal((n_sc, U, B)) + 1j * g_h.standard_normal((n_sc, U, B))) / np.sqrt(2.0)
    if corr_r is not None:
        Lr = np.linalg.cholesky(exp_correlation(B, corr_r))      # R = Lr Lr^T
        H = H @ Lr.T                      # per user: h_u <- R^{1/2} h_u (antennas contiguous)
    H = H.astype(np.complex64)

    L, e_avg = qam_levels(bits)
    levels = g_s.integers(0, L, size=(n_sc, n_sym, U, 2)).astype(np.int8)
    amp = (2.0 * levels.astype(np.float64) - (L - 1)) * np.sqrt(Es / e_avg)
    s = amp[..., 0] + 1j * amp[..., 1]

    N0 = 0.0 if noiseless else noise_variance(U, Es, snr_db)
    # y[k][n][b] = sum_u H[k][u][b] s[k][n][u] + noise, formed in float64 from the
    # complex64-rounded channel, then rounded once to complex64.
    y = s @ H.astype(np.complex128)   # [n_sc][n_sym][U] @ [n_sc][U][B]
    if not noiseless:
        y = y + np.sqrt(N0 / 2.0) * (g_n.standard_normal(y.shape) + 1j * g_n.standard_normal(y.shape))
    y = y.astype(np.complex64)
    return Problem(H=H, y=y, s=s, levels=levels, N0=N0, Es=float(Es), B=B, U=U, C=C,
                   n_sc=n_sc, n_sym=n_sym, bits=bits, snr_db=float(snr_db))


def make_uneven(n_inst: int, *, seed: int = 0, U_range=(4, 32), B_choices=(64, 128, 256),
                C_choices=(1, 2, 4, 8, 16), nsym_range=(1, 14), snr_range=(5.0, 20.0), bits: int = 4,
                n_sc: int = 1, min_S: int = 4) -> list[Problem]:
    """Draw ``n_inst`` independent problems of uneven size (one seeded stream for
    the sizes, one ``make_problem`` seed per instance).

    Per instance: U uniform on ``U_range`` (inclusive), B from ``B_choices``, C
    from the ``C_choices`` that divide B with at least ``min_S`` antennas per
    cluster, n_sym uniform on ``nsym_range`` (inclusive), SNR uniform on
    ``snr_range`` dB, ``bits``-bit square QAM, i.i.d. CN(0, 1) channels.
    """
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x5EED])))
    out = []
    for i in range(n_inst):
        U = int(g.integers(U_range[0], U_range[1] + 1))
        B = int(g.choice(B_choices))
        Cs = [c for c in C_choices if B % c == 0 and B // c >= min_S]
        C = int(g.choice(Cs))
        n_sym = int(g.integers(nsym_range[0], nsym_range[1] + 1))
        snr = float(g.uniform(*snr_range))
        out.append(make_problem(B, U, C, n_sc, n_sym, snr_db=snr, bits=bits, seed=seed * 1_000_003 + i))
    return out
