"""Pins of the FP64 LAMA oracle (Sec. III-B, Algorithm 1, Eq. F, Thm. 2, Lemma 5) — CPU only.

Each test checks the oracle against something other than itself: the closed
form of the QPSK posterior mean, the limits of the denoiser, the original
centralized LAMA of the derivation in Appendix A (iterating on the B-dimensional
residual instead of the Gram matrix), the state-evolution recursion of Thm. 2
and Lemma 5 (evaluated by Gauss-Hermite quadrature) against Monte-Carlo MSEs,
and exact recovery at high SNR.
"""
import numpy as np
import pytest

from oracle import lama
from paper_1808_04473_gb300 import synth


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_qpsk_denoiser_is_the_tanh_posterior_mean():
    """QPSK: per axis the posterior of +-a under N(0, tau/2) noise has mean a tanh(2 a x / tau)."""
    Es, tau = 1.7, 0.37
    pts = lama.qam_points(2, Es)
    a = np.sqrt(Es / 2)
    rng = np.random.default_rng(0)
    z = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    F, G = lama.denoise(z, tau, pts)
    Fr, Fi = a * np.tanh(2 * a * z.real / tau), a * np.tanh(2 * a * z.imag / tau)
    np.testing.assert_allclose(F, Fr + 1j * Fi, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(G, 2 * a * a - Fr ** 2 - Fi ** 2, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("bits", [2, 4, 6])
def test_denoiser_limits(bits):
    """tau -> inf: the prior's mean 0 and variance Es; tau -> 0: the nearest point, variance 0."""
    Es = 1.3
    pts = lama.qam_points(bits, Es)
    assert np.mean(np.abs(pts) ** 2) == pytest.approx(Es, rel=1e-12)
    rng = np.random.default_rng(bits)
    z = 0.5 * (rng.standard_normal(40) + 1j * rng.standard_normal(40))
    F, G = lama.denoise(z, 1e9, pts)
    assert np.abs(F).max() < 1e-6 and np.allclose(G, Es, rtol=1e-6)
    F, G = lama.denoise(z, 1e-6, pts)
    near = pts[np.argmin(np.abs(z[:, None] - pts[None, :]), axis=1)]
    np.testing.assert_allclose(F, near, atol=1e-9)
    assert G.max() < 1e-9


def _centralized_lama(Hm, y, N0, Es, points, T):
    """The original LAMA on (H, y) as the derivation of Algorithm 1 (Appendix A) starts from,
    on the paper's normalization (H entries of variance 1/B): residual r in C^B."""
    B, U = Hm.shape
    H = Hm / np.sqrt(B)
    yv = y / np.sqrt(B)
    N0p, beta = N0 / B, U / B
    s = np.zeros(U, np.complex128)
    tau = beta * Es / N0p                               # phi^1 = Es, tau = beta phi / N0
    r = yv - H @ s
    for t in range(1, T + 1):
        z = s + H.conj().T @ r
        if t == T:
            return z, N0p * (1 + tau)
        s, g = lama.denoise(z, N0p * (1 + tau), points)
        tau_new = beta / N0p * np.mean(g)
        r = yv - H @ s + tau_new / (1 + tau) * r
        tau = tau_new


@pytest.mark.parametrize("bits,T", [(2, 1), (2, 6), (4, 8), (6, 5)])
def test_lama_pd_equals_the_centralized_lama(bits, T):
    """Algorithm 1 on (G, y^MRC) gives the same iterates as LAMA on (H, y) (Sec. III-B)."""
    p = synth.make_problem(64, 8, 4, 3, 2, snr_db=12.0, bits=bits, seed=40 + T)
    o = lama.equalize_pd_lama(p.H, p.y, p.N0, p.Es, 4, bits, T)
    pts = lama.qam_points(bits, p.Es)
    for k in range(p.H.shape[0]):
        Hm = p.H[k].astype(np.complex128).T
        for n in range(p.y.shape[1]):
            z, s2 = _centralized_lama(Hm, p.y[k, n].astype(np.complex128), p.N0, p.Es, pts, T)
            assert _rel(o["z"][k, n], z) < 1e-10
            assert o["sigma2"][k, n, 0] == pytest.approx(s2, rel=1e-10)


def test_one_iteration_is_the_normalized_matched_filter():
    """T = 1: z^1 = y^MRC / B with sigma_1^2 = N0/B + beta Es (the initial value of Thm. 2)."""
    p = synth.make_problem(32, 4, 2, 3, 2, snr_db=5.0, bits=4, seed=41)
    o = lama.equalize_pd_lama(p.H, p.y, p.N0, p.Es, 2, 4, 1)
    for k in range(3):
        Hm = p.H[k].astype(np.complex128)
        ymr = (Hm.conj() @ p.y[k].astype(np.complex128).T) / 32
        np.testing.assert_allclose(o["z"][k], ymr.T, rtol=1e-12)
    np.testing.assert_allclose(o["sigma2"], p.N0 / 32 + 4 / 32 * p.Es, rtol=1e-12)


def test_fd_equals_pd_for_one_cluster():
    p = synth.make_problem(48, 6, 1, 3, 3, snr_db=8.0, bits=4, seed=42)
    pd = lama.equalize_pd_lama(p.H, p.y, p.N0, p.Es, 1, 4, 5)
    fd = lama.equalize_fd_lama(p.H, p.y, p.N0, p.Es, 1, 4, 5)
    assert _rel(fd["z"], pd["z"]) < 1e-12 and _rel(fd["sigma2"], pd["sigma2"]) < 1e-12


def _psi(sigma2, bits, Es, nodes=80):
    """MSE function of Thm. 2, E|F(S + sigma Z, sigma^2) - S|^2, by Gauss-Hermite quadrature:
    square QAM factorizes into two PAM axes with noise N(0, sigma^2/2) each."""
    x, w = np.polynomial.hermite_e.hermegauss(nodes)
    w = w / np.sqrt(2 * np.pi)
    pts = lama.qam_points(bits, Es)
    lev = np.unique(np.round(pts.real, 12))
    tot = 0.0
    for a in lev:
        F, _ = lama.denoise(a + np.sqrt(sigma2 / 2) * x + 0j, sigma2, pts)
        tot += np.sum(w * (F.real - a) ** 2)
    return 2.0 * tot / len(lev)


@pytest.mark.slow
@pytest.mark.parametrize("bits,snr_db", [(2, 4.0), (4, 10.0)])
def test_state_evolution_predicts_the_mse_of_every_iteration(bits, snr_db):
    """Thm. 2: sigma_t^2 = N0 + beta Psi(sigma_{t-1}^2), sigma_1^2 = N0 + beta Es, is the MSE of
    z^t (large system: B = 256, U = 32; 4000 vectors).  The variance the algorithm reports,
    N0 + beta phi^t, tracks it too."""
    B, U, T = 256, 32, 6
    p = synth.make_problem(B, U, 1, 250, 16, snr_db=snr_db, bits=bits, seed=43)
    N0n, beta = p.N0 / B, U / B
    se = [N0n + beta * p.Es]
    for _ in range(T - 1):
        se.append(N0n + beta * _psi(se[-1], bits, p.Es))
    for t in range(1, T + 1):
        o = lama.equalize_pd_lama(p.H, p.y, p.N0, p.Es, 1, bits, t)
        mse = np.mean(np.abs(o["z"] - p.s) ** 2)
        assert mse == pytest.approx(se[t - 1], rel=0.03), (t, mse, se[t - 1])
        assert np.mean(o["sigma2"]) == pytest.approx(se[t - 1], rel=0.03)


@pytest.mark.slow
def test_fd_fused_variance_follows_lemma5_and_thm3():
    """LAMA-FD: per cluster w_c sigma_c^2 = N0 + beta Psi(sigma_c^2) (Lemma 5, iterated as the
    cluster's state evolution), fused sigma^2 = (sum_c sigma_c^-2)^-1 (Thm. 3) is the MSE of
    the fused estimate; unequal clusters (3/4, 1/4)."""
    B, U, T, bits = 256, 16, 6, 4
    sizes = [192, 64]
    p = synth.make_problem(B, U, 2, 200, 16, snr_db=8.0, bits=bits, seed=44)
    o = lama.equalize_fd_lama(p.H, p.y, p.N0, p.Es, 2, bits, T, cluster_sizes=sizes)
    inv = 0.0
    for S in sizes:
        s2 = p.N0 / S + U / S * p.Es
        for _ in range(T - 1):
            s2 = p.N0 / S + U / S * _psi(s2, bits, p.Es)
        inv += 1.0 / s2
    mse = np.mean(np.abs(o["z"] - p.s) ** 2)
    assert mse == pytest.approx(1.0 / inv, rel=0.08)
    assert np.mean(o["sigma2"]) == pytest.approx(1.0 / inv, rel=0.08)


def test_high_snr_recovers_the_symbols():
    p = synth.make_problem(128, 16, 2, 6, 8, snr_db=25.0, bits=4, seed=45)
    pts = lama.qam_points(4, p.Es)
    for f in (lama.equalize_pd_lama, lama.equalize_fd_lama):
        o = f(p.H, p.y, p.N0, p.Es, 2, 4, 8)
        hard = pts[np.argmin(np.abs(o["z"][..., None] - pts), axis=-1)]
        assert np.abs(hard - p.s).max() < 1e-5


def test_lama_needs_noise():
    p = synth.make_problem(32, 4, 2, 2, 1, noiseless=True, seed=46)
    with pytest.raises(ValueError):
        lama.equalize_pd_lama(p.H, p.y, 0.0, p.Es, 2, 4, 3)
