"""Pins of the FP64 MRC and ZF oracle (Sec. III-A definitions, FD per Sec. IV-A) — CPU only.

Each test checks the oracle against something other than itself: SVD least
squares for ZF, a per-user loop for MRC, the statistical meaning of the error
variances (Monte Carlo), noiseless recovery, and the complex Wishart moment
behind Lemma 4's FD-ZF SINR.
"""
import numpy as np
import pytest

from oracle import linear, lmmse
from paper_1808_04473_gb300 import synth


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("seed,B,U,C", [(0, 8, 3, 2), (1, 12, 5, 3), (2, 6, 6, 1), (3, 64, 16, 8)])
def test_pd_zf_equals_least_squares(seed, B, U, C):
    """PD-ZF ``G^{-1} y^MRC`` is the least-squares solution of ``y = H s`` (SVD, no Gram matrix)."""
    p = synth.make_problem(B, U, C, 4, 3, snr_db=7.0, seed=seed)
    o = linear.equalize_pd_linear(p.H, p.y, p.N0, p.Es, C, "zf")
    for k in range(p.H.shape[0]):
        Hm = p.H[k].astype(np.complex128).T
        ls = np.linalg.lstsq(Hm, p.y[k].astype(np.complex128).T, rcond=None)[0]
        assert _rel(o["z"][k].T, ls) < 1e-10
    assert not o["info"].any()


@pytest.mark.parametrize("C", [1, 2, 4])
def test_pd_mrc_is_the_per_user_matched_filter(C):
    """PD-MRC: ``z_u = h_u^H y / ||h_u||^2`` user by user; the variance by brute-force sums."""
    p = synth.make_problem(16, 5, C, 3, 4, snr_db=5.0, seed=4)
    o = linear.equalize_pd_linear(p.H, p.y, p.N0, p.Es, C, "mrc")
    for k in range(p.H.shape[0]):
        h = p.H[k].astype(np.complex128)                       # U x B: row u is h_u
        for u in range(h.shape[0]):
            nu = np.vdot(h[u], h[u]).real
            for t in range(p.y.shape[1]):
                zu = np.vdot(h[u], p.y[k, t].astype(np.complex128)) / nu
                assert abs(o["z"][k, t, u] - zu) < 1e-12 * max(1.0, abs(zu))
            interf = sum(abs(np.vdot(h[u], h[v])) ** 2 for v in range(h.shape[0]) if v != u)
            s2 = p.N0 / nu + p.Es * interf / nu ** 2
            assert o["sigma2"][k, u] == pytest.approx(s2, rel=1e-12)


@pytest.mark.parametrize("equalizer", ["mrc", "zf"])
def test_error_variances_are_the_mean_squared_errors(equalizer):
    """sigma^2 is E|z_u - s_u|^2 given H (Sec. II-A) and both estimates are unbiased."""
    B, U, n = 16, 4, 40000
    p = synth.make_problem(B, U, 1, 1, n, snr_db=3.0, seed=8, bits=2)
    o = linear.equalize_pd_linear(p.H, p.y, p.N0, p.Es, 1, equalizer)
    z, s = o["z"][0].T, p.s[0].T                                 # U x n
    emp = np.mean(np.abs(z - s) ** 2, axis=1)
    np.testing.assert_allclose(emp, o["sigma2"][0], rtol=0.04)
    gain = np.real(np.mean(np.conj(s) * z, axis=1)) / p.Es
    np.testing.assert_allclose(gain, 1.0, atol=0.03)


@pytest.mark.parametrize("equalizer", ["mrc", "zf"])
def test_fd_equals_pd_for_one_cluster(equalizer):
    p = synth.make_problem(24, 5, 1, 4, 3, seed=6)
    pd = linear.equalize_pd_linear(p.H, p.y, p.N0, p.Es, 1, equalizer)
    fd = linear.equalize_fd_linear(p.H, p.y, p.N0, p.Es, 1, equalizer)
    assert _rel(fd["z"], pd["z"]) < 1e-12
    assert _rel(fd["sigma2"], pd["sigma2"]) < 1e-12


def test_fd_zf_fused_variance_is_the_fused_mean_squared_error():
    """FD-ZF: the cluster errors are pure noise on disjoint antennas, hence independent,
    and the fused variance of Thm. 3 is exactly the MSE of the fused estimate (Lemma 1)."""
    B, U, C, n = 32, 4, 4, 30000
    p = synth.make_problem(B, U, C, 1, n, snr_db=2.0, seed=12, bits=2)
    o = linear.equalize_fd_linear(p.H, p.y, p.N0, p.Es, C, "zf")
    emp = np.mean(np.abs(o["z"][0] - p.s[0]) ** 2, axis=0)
    np.testing.assert_allclose(emp, o["sigma2"][0], rtol=0.04)


def test_fd_mrc_fuses_the_per_cluster_matched_filters():
    """FD-MRC: each cluster's pair is PD-MRC on that cluster alone (pinned above by a per-user
    loop), fused with weights ``(1/sigma2_c) / sum_c' (1/sigma2_c')`` (Eq. opt_fusion); the fused
    estimate is unbiased.  Its reported variance is Thm. 3's model value: the clusters'
    interference terms share ``s`` and are correlated, so it is not the exact MSE given ``H``."""
    B, U, C, n = 32, 4, 4, 20000
    sizes = [4, 12, 10, 6]
    p = synth.make_problem(B, U, C, 1, n, snr_db=2.0, seed=17, bits=2)
    o = linear.equalize_fd_linear(p.H, p.y, p.N0, p.Es, C, "mrc", cluster_sizes=sizes)
    zs, inv, b0 = [], [], 0
    for bc in sizes:
        c = linear.equalize_pd_linear(p.H[:, :, b0:b0 + bc], p.y[:, :, b0:b0 + bc], p.N0, p.Es, 1, "mrc")
        zs.append(c["z"][0])
        inv.append(1.0 / c["sigma2"][0])
        b0 += bc
    inv = np.array(inv)
    zf = sum(inv[c][None, :] * zs[c] for c in range(C)) / inv.sum(axis=0)[None, :]
    assert _rel(o["z"][0], zf) < 1e-12
    np.testing.assert_allclose(o["sigma2"][0], 1.0 / inv.sum(axis=0), rtol=1e-12)
    gain = np.real(np.mean(np.conj(p.s[0]) * o["z"][0], axis=0)) / p.Es
    np.testing.assert_allclose(gain, 1.0, atol=0.03)


@pytest.mark.parametrize("arch", ["pd", "fd"])
def test_noiseless_zf_recovers_the_symbols(arch):
    p = synth.make_problem(32, 4, 2, 5, 3, noiseless=True, seed=9)
    f = linear.equalize_pd_linear if arch == "pd" else linear.equalize_fd_linear
    o = f(p.H, p.y, 0.0, p.Es, 2, "zf")
    assert np.abs(o["z"] - p.s).max() < 1e-5
    assert np.all(o["sigma2"] == 0.0)


def test_noiseless_single_user_mrc_recovers_the_symbol():
    """U = 1: MRC has no interference; with N0 = 0 it recovers s and has variance 0."""
    p = synth.make_problem(16, 1, 4, 3, 5, noiseless=True, seed=13)
    for f in (linear.equalize_pd_linear, linear.equalize_fd_linear):
        o = f(p.H, p.y, 0.0, p.Es, 4, "mrc")
        assert np.abs(o["z"] - p.s).max() < 1e-5
        assert np.all(o["sigma2"] == 0.0)


def test_fd_zf_sinr_has_the_complex_wishart_mean():
    """FD-ZF: ``1/sigma2_u = sum_c 1/(N0 [G_c^{-1}]_uu)`` with ``1/[G_c^{-1}]_uu ~ Gamma(S_c-U+1)``
    for i.i.d. CN(0,1) channels, so ``E[Es/sigma2] = (Es/N0)(B - C(U-1))`` — the finite-size
    form of Lemma 4, which reaches ``(Es/N0)(1 - C beta) B`` as ``B -> infinity``.
    A wrong diagonal (``[G_c]_uu`` instead of ``[G_c^{-1}]_uu``) or fusion gives ``B`` or ``C`` times off."""
    B, U, C, n_sc = 32, 4, 4, 1500
    p = synth.make_problem(B, U, C, n_sc, 1, snr_db=10.0, seed=14)
    o = linear.equalize_fd_linear(p.H, p.y, p.N0, p.Es, C, "zf")
    mean = np.mean(p.Es / o["sigma2"])
    expect = p.Es / p.N0 * (B - C * (U - 1))
    assert mean == pytest.approx(expect, rel=0.02)


def test_zf_singular_cluster_reports_first_nonpositive_minor():
    """A user that one cluster cannot see makes that ``G_c`` singular at the user's index:
    ZF reports it (1-based) and that subcarrier's outputs are NaN; MRC needs no inverse."""
    p = synth.make_problem(16, 4, 2, 3, 2, seed=15)
    H = p.H.copy()
    H[1, 2, :8] = 0.0                                            # user 2, cluster 0, subcarrier 1
    o = linear.equalize_fd_linear(H, p.y, p.N0, p.Es, 2, "zf")
    assert o["info"].tolist() == [[0, 0], [3, 0], [0, 0]]
    assert np.isnan(o["z"][1]).all() and np.isfinite(o["z"][[0, 2]]).all()
    o = linear.equalize_fd_linear(H, p.y, p.N0, p.Es, 2, "mrc")
    assert np.isfinite(o["z"]).all() and not o["info"].any()


def test_invisible_user_gets_zero_mrc_weight():
    p = synth.make_problem(16, 3, 2, 2, 2, seed=11)
    H = p.H.copy()
    H[0, 1, :8] = 0.0                                            # user 1 unseen by cluster 0
    o = linear.equalize_fd_linear(H, p.y, p.N0, p.Es, 2, "mrc")
    one = linear.equalize_pd_linear(H[:, :, 8:], p.y[:, :, 8:], p.N0, p.Es, 1, "mrc")
    np.testing.assert_allclose(o["z"][0, :, 1], one["z"][0, :, 1], rtol=1e-12)
    assert o["sigma2"][0, 1] == pytest.approx(one["sigma2"][0, 1], rel=1e-12)


def test_lmmse_beats_zf_and_mrc_in_mean_squared_error():
    """L-MMSE minimizes the MSE among linear equalizers (Sec. III-A): per user, its biased
    error variance is at most ZF's and MRC's on the same channel."""
    p = synth.make_problem(16, 6, 1, 8, 1, snr_db=4.0, seed=16)
    lm = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, 1, "literal")
    for eq in ("mrc", "zf"):
        o = linear.equalize_pd_linear(p.H, p.y, p.N0, p.Es, 1, eq)
        assert np.all(lm["sigma2"] <= o["sigma2"] * (1 + 1e-12))


def _disjoint_users(seed):
    """U = 3 on B = 64 antennas, C = 4 clusters of 16, noise at 10 dB: clusters 0 and 1
    see user 0 alone, cluster 2 all three users, cluster 3 users 1 and 2.  Read with
    N0 = 0, user 0 has no interference in clusters 0 and 1 (variance exactly 0 there)
    and users 1 and 2 have interference in every cluster that sees them."""
    p = synth.make_problem(64, 3, 4, 4, 2, snr_db=10.0, seed=seed)
    n = p.y.astype(np.complex128) - p.s @ p.H.astype(np.complex128)
    H = p.H.copy()
    H[:, 1:, :32] = 0.0
    H[:, 0, 48:] = 0.0
    y = (p.s @ H.astype(np.complex128) + n).astype(np.complex64)
    return p, H, y


def test_mrc_zero_variance_pairs_take_the_limit_weights():
    """Lemma 1's weights sigma_c^-2 / sum sigma^-2 as N0 -> 0.  FD: the outputs for
    N0 = 1e-6, 1e-9, 1e-12 (ordinary weights: no variance is 0 there) converge
    linearly in N0 to the N0 = 0 output, in which user 0's two zero-variance clusters
    share the weight in proportion to G_c,uu, i.e. z_0 = sum_{b < 32} conj(h_0b) y_b /
    sum_{b < 32} |h_0b|^2 (written out here per antenna), with variance 0, and users
    1 and 2 keep the ordinary weights.  PD (no fusion step, z = y^MRC_u / G_uu) does
    not depend on N0."""
    p, H, y = _disjoint_users(18)
    for f in (linear.equalize_pd_linear, linear.equalize_fd_linear):
        lim = f(H, y, 0.0, p.Es, 4, "mrc")
        for N0 in (1e-6, 1e-9, 1e-12):
            o = f(H, y, N0, p.Es, 4, "mrc")
            assert (o["sigma2"] > 0).all()
            assert np.abs(o["z"] - lim["z"]).max() <= 10 * N0, (f.__name__, N0)
            assert np.abs(o["sigma2"] - lim["sigma2"]).max() <= 10 * N0, (f.__name__, N0)
        assert (lim["sigma2"][:, 1:] > 0).all()
    fd = linear.equalize_fd_linear(H, y, 0.0, p.Es, 4, "mrc")
    for k in range(p.n_sc):
        for n in range(p.n_sym):
            num = sum(np.conj(complex(H[k, 0, b])) * complex(y[k, n, b]) for b in range(32))
            den = sum(abs(complex(H[k, 0, b])) ** 2 for b in range(32))
            assert abs(fd["z"][k, n, 0] - num / den) < 1e-12
    assert (fd["sigma2"][:, 0] == 0).all()
    # Reading the pair with variance 0 as weight 0 would drop clusters 0 and 1.
    assert np.abs(fd["z"][:, :, 0]).min() > 0.1


def test_mrc_zero_variance_pd_equals_fd_at_c1():
    """PD and FD at C = 1 agree in the zero-variance case too (one pair, weight 1)."""
    p = synth.make_problem(32, 2, 1, 3, 2, noiseless=True, seed=18)
    H = p.H.copy()
    H[:, 0, 16:] = 0.0
    H[:, 1, :16] = 0.0
    y = np.einsum("kub,knu->knb", H.astype(np.complex128), p.s).astype(np.complex64)
    pd = linear.equalize_pd_linear(H, y, 0.0, p.Es, 1, "mrc")
    fd = linear.equalize_fd_linear(H, y, 0.0, p.Es, 1, "mrc")
    assert _rel(fd["z"], pd["z"]) < 1e-14 and np.array_equal(pd["sigma2"], fd["sigma2"])
    np.testing.assert_allclose(pd["z"], p.s, atol=1e-12)
    assert (pd["sigma2"] == 0).all()


@pytest.mark.slow
def test_large_system_mrc_matches_cor1_and_fd_equals_pd():
    """Cor. 1: MRC reaches SINR = snr / (1 + beta snr) (paper normalization, snr = B Es / N0 here);
    Lemma 8: FD-MRC fused with the optimal weights equals PD-MRC.  B = 1024, U = 64, C = 8:
    the empirical Es / MSE of both within 0.2 dB of the closed form (the finite-size
    interference of U - 1 users instead of U is 0.07 dB)."""
    from oracle import theory
    B, U, C = 1024, 64, 8
    p = synth.make_problem(B, U, C, 30, 16, snr_db=10.0, bits=4, seed=19)
    expect = theory.db(theory.sinr_pd("mrc", U / B, B * p.Es / p.N0))
    for f in (linear.equalize_pd_linear, linear.equalize_fd_linear):
        o = f(p.H, p.y, p.N0, p.Es, C, "mrc")
        emp = theory.db(p.Es / np.mean(np.abs(o["z"] - p.s) ** 2))
        assert abs(emp - expect) < 0.2, (f.__name__, emp, expect)


def test_zf_variance_has_the_inverse_wishart_mean():
    """PD-ZF: E[(G^{-1})_uu] = 1 / (B - U) for i.i.d. CN(0, 1) channels, so the mean reported
    variance is N0 / (B - U) — Cor. 1's SINR snr (1 - beta) in the paper's normalization."""
    B, U = 64, 8
    p = synth.make_problem(B, U, 1, 800, 1, snr_db=10.0, seed=20)
    o = linear.equalize_pd_linear(p.H, p.y, p.N0, p.Es, 1, "zf")
    assert np.mean(o["sigma2"]) == pytest.approx(p.N0 / (B - U), rel=0.02)
