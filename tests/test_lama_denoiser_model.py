"""The LAMA kernel's denoiser formulation, modelled in float32 on the host (CPU only).

The kernel computes the posterior of Eq. F per PAM axis: the 2-D posterior of a
square constellation under circular Gaussian noise factorizes into two axes with
noise variance tau / 2 each.  Exponents are taken relative to the nearest level
a0 and the moments about a0.  This test restates that formulation in float32
NumPy.  It checks it against the oracle's FP64 brute force over every
constellation point, including the regimes the GPU parity cases reach only
rarely: tau from 1e-6 to 1e6, points far outside the constellation, and sharp
posteriors on the outer levels, where E[a^2] - E[a]^2 would cancel.  The bound
is a few times the change that float32 rounding of z, and of the exponents'
arguments, makes to the exact posterior: near a decision boundary with small
tau any float32 evaluation is ill-conditioned, elsewhere the bound is 1e-6.
"""
import numpy as np
import pytest

from oracle import lama


def _axis_model(x, tau, d, L):
    """Float32 posterior mean and variance of one axis, as the kernel forms them."""
    f = np.float32
    x = x.astype(f)
    l2t = f(np.log2(np.e)) * (f(1.0) / f(tau))             # log2(e) / tau: the weights in base 2
    inv_d = f(1.0) / f(d)
    q = np.clip(np.rint((x * inv_d + f(L - 1)) * f(0.5)), 0, L - 1).astype(f)
    a0 = (f(2) * q - f(L - 1)) * f(d)
    e0 = (x - a0) * (x - a0)
    sw = np.zeros_like(x)
    s1 = np.zeros_like(x)
    s2 = np.zeros_like(x)
    for m in range(L):
        a = (f(2 * m) - f(L - 1)) * f(d)
        e = x - a
        w = np.exp2((e0 - e * e) * l2t).astype(f)
        da = a - a0
        sw += w
        s1 += w * da
        s2 += w * da * da
    m1 = s1 / sw
    return a0 + m1, np.maximum(s2 / sw - m1 * m1, f(0))


@pytest.mark.parametrize("bits", [2, 4, 6, 8])
@pytest.mark.parametrize("tau", [1e-6, 1e-3, 0.05, 1.0, 1e3, 1e6])
def test_axis_factorization_matches_the_2d_posterior(bits, tau):
    Es = 1.0
    L = 1 << (bits // 2)
    d = np.sqrt(Es / (2.0 * (L * L - 1) / 3.0))
    pts = lama.qam_points(bits, Es)
    rng = np.random.default_rng(bits * 7 + int(np.log10(tau) + 7))
    lev = (2 * np.arange(L) - (L - 1)) * d
    z = np.concatenate([
        rng.normal(0, 1.5 * L * d, 64) + 1j * rng.normal(0, 1.5 * L * d, 64),   # across and beyond the grid
        lev[-1] + 1e-3 * d + 1j * (lev[0] - 1e-3 * d) + 0 * np.arange(4),      # sharp on outer levels
        0.5 * (lev[0] + lev[1]) + 1j * 0.5 * (lev[-2] + lev[-1]) + 0 * np.arange(4),  # on decision boundaries
        40.0 * L * d * (1 + 1j) + 0 * np.arange(2),                              # far outside
    ])
    z = z.astype(np.complex64).astype(np.complex128)        # the kernel's inputs are float32
    F, G = lama.denoise(z, tau, pts)
    mr, vr = _axis_model(z.real, tau, d, L)
    mi, vi = _axis_model(z.imag, tau, d, L)
    # Bound: a few times what a float32 rounding of z moves the exact posterior by (the
    # condition of F and G at z; near a decision boundary with small tau it is large
    # for any float32 evaluation), plus 1e-6 of the constellation's scale.
    eps = 2.0 ** -24 * (np.abs(z.real) + np.abs(z.imag) + d)
    Fp, Gp = lama.denoise(z + eps * (1 + 1j), tau, pts)
    Fm, Gm = lama.denoise(z - eps * (1 + 1j), tau, pts)
    # ... and what float32 rounding of the exponents' arguments (x - a)^2 / tau does where a
    # second level carries weight: a relative error delta of its weight w2 moves the
    # mean by about d delta w2 and the variance by about d^2 delta w2.
    term = np.zeros(z.shape)
    for x in (z.real, z.imag):
        dist = np.sort(np.abs(x[:, None] - lev[None, :]), axis=1)
        w2 = np.exp(-(dist[:, 1] ** 2 - dist[:, 0] ** 2) / tau)
        term += 4 * 2.0 ** -24 * dist[:, 1] ** 2 / tau * np.minimum(w2, 1.0)
    tolF = 8 * np.abs(Fp - Fm) + 4 * d * term + 1e-6 * np.sqrt(Es)
    tolG = 8 * np.abs(Gp - Gm) + 8 * d * d * term + 1e-6 * Es
    assert (np.abs((mr + 1j * mi) - F) <= tolF).all()
    assert (np.abs((vr + vi) - G) <= tolG).all()
    well = (tolF < 1e-5) & (tolG < 1e-5)                       # most points: well conditioned
    assert well.mean() > 0.5
