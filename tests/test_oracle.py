"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a different
algorithm (SVD least squares), an algebraic identity, the statistical meaning
of a quantity (Monte-Carlo error variances), a closed form from the paper's
large-system analysis, or a value printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import llr, lmmse, theory
from paper_1808_04473_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------------------- exact pins

@pytest.mark.parametrize("seed,B,U,C,Es", [(0, 8, 3, 2, 1.0), (1, 12, 5, 3, 2.5), (2, 6, 6, 1, 0.7),
                                          (3, 16, 4, 4, 1.0), (4, 4, 7, 2, 1.3)])
def test_pd_equals_regularized_least_squares(seed, B, U, C, Es):
    """PD L-MMSE (Sec. III-A) equals argmin ||y-Hx||^2 + rho||x||^2 solved by SVD (no Gram matrix)."""
    p = synth.make_problem(B, U, C, 5, 3, snr_db=7.0, seed=seed, Es=Es)
    pd = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, C, "literal")
    ls = lmmse.centralized_lmmse(p.H, p.y, p.N0, p.Es)
    assert _rel(pd["z"], ls) < 1e-11


def test_pd_is_independent_of_the_partition():
    """PD gives exactly the centralized estimates for every C (Sec. III-A, last paragraph)."""
    p = synth.make_problem(64, 6, 1, 4, 2, seed=5)
    ref = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, 1)
    for C in (2, 4, 8, 16, 64):
        o = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, C)
        assert _rel(o["z"], ref["z"]) < 1e-12
        assert _rel(o["sigma2"], ref["sigma2"]) < 1e-12
    o = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, 3, cluster_sizes=[10, 30, 24])
    assert _rel(o["z"], ref["z"]) < 1e-12


@pytest.mark.parametrize("estimate", ["literal", "unbiased"])
def test_pd_equals_fd_for_one_cluster(estimate):
    """With C=1 the two architectures coincide (Lemma 3, equality case C=1)."""
    p = synth.make_problem(24, 5, 1, 6, 3, seed=6)
    pd = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, 1, estimate)
    fd = lmmse.equalize_fd(p.H, p.y, p.N0, p.Es, 1, estimate)
    assert _rel(fd["z"], pd["z"]) < 1e-12
    assert _rel(fd["sigma2"], pd["sigma2"]) < 1e-12


def test_literal_error_variance_reduces_to_N0_diag_inverse():
    """With rho = N0/Es, diag(A G A^H N0 + (AG-I)(AG-I)^H Es) = N0 diag(A) (A G = I - rho A)."""
    rng = np.random.default_rng(7)
    for U, B in ((4, 9), (16, 32), (8, 5)):
        Hm = (rng.standard_normal((B, U)) + 1j * rng.standard_normal((B, U)))
        G = Hm.conj().T @ Hm
        N0, Es = 0.37, 1.9
        z, s2, A, mu, info = lmmse.lmmse_unit(G, np.zeros((U, 1)), N0, Es)
        assert info == 0
        np.testing.assert_allclose(s2, N0 * np.real(np.diag(A)), rtol=1e-10)
        np.testing.assert_allclose(mu, 1.0 - N0 / Es * np.real(np.diag(A)), rtol=1e-10)


def test_error_variances_are_the_mean_squared_errors():
    """sigma^2 is E|z - s0|^2 given H (Sec. II-A); the unbiased pair matches E|z/mu - s0|^2.

    Fixed channel, 40000 independent (s0, n) draws; the empirical per-user MSE
    must match the formula within Monte-Carlo error (about 1%).
    """
    B, U, n = 12, 6, 40000
    p = synth.make_problem(B, U, 1, 1, n, snr_db=3.0, seed=8, bits=2)
    Hm = p.H[0].astype(np.complex128).T
    G, yMR = lmmse.local_preprocess(Hm, p.y[0].astype(np.complex128).T)
    z, s2, A, mu, _ = lmmse.lmmse_unit(G, yMR, p.N0, p.Es)
    s = p.s[0].T                                                        # U x n
    emp = np.mean(np.abs(z - s) ** 2, axis=1)
    np.testing.assert_allclose(emp, s2, rtol=0.04)
    zu, s2u = lmmse.unbias(z, s2, mu, p.Es)
    emp_u = np.mean(np.abs(zu - s) ** 2, axis=1)
    np.testing.assert_allclose(emp_u, s2u, rtol=0.04)
    np.testing.assert_allclose(s2u, s2 / mu, rtol=1e-10)                # L-MMSE: sigma2_u = sigma2/mu
    gain = np.real(np.mean(np.conj(s) * zu, axis=1)) / p.Es
    np.testing.assert_allclose(gain, 1.0, atol=0.03)                   # unbiased


@pytest.mark.parametrize("arch", ["pd", "fd"])
def test_noiseless_zero_forcing_recovers_the_symbols(arch):
    """N0 = 0 makes L-MMSE the ZF equalizer (Sec. III-A), exact when H (or each H_c) has full column rank."""
    p = synth.make_problem(32, 4, 2, 8, 3, noiseless=True, seed=9)
    f = lmmse.equalize_pd if arch == "pd" else lmmse.equalize_fd
    o = f(p.H, p.y, 0.0, p.Es, 2)
    assert np.abs(o["z"] - p.s).max() < 1e-5      # inputs are complex64-rounded: y = H s rounded once
    assert np.all(np.abs(o["sigma2"]) < 1e-20)       # exactly zero up to FP64 rounding


def test_singular_system_reports_first_nonpositive_minor():
    """ZF on a channel with an all-zero user column: G + 0 I is singular at that user's index."""
    p = synth.make_problem(16, 4, 2, 3, 2, noiseless=True, seed=10)
    H = p.H.copy()
    H[1, 2, :] = 0.0
    o = lmmse.equalize_pd(H, p.y, 0.0, p.Es, 2)
    assert list(o["info"]) == [0, 3, 0]
    assert np.isnan(o["z"][1]).all() and np.isfinite(o["z"][0]).all()
    M = np.diag([1.0, 2.0, -1.0, 3.0])
    assert lmmse.first_nonpositive_minor(M) == 3
    assert lmmse.first_nonpositive_minor(np.eye(5)) == 0


def test_zero_column_with_regularization_gets_zero_weight():
    """rho > 0 and H_c[:, u] = 0: mu = 0, infinite unbiased variance, zero fusion weight."""
    p = synth.make_problem(16, 3, 2, 2, 2, seed=11)
    H = p.H.copy()
    H[0, 1, :8] = 0.0                           # user 1 invisible to cluster 0 on subcarrier 0
    o = lmmse.equalize_fd(H, p.y, p.N0, p.Es, 2)
    assert o["nu"][0, 0, 1] == 0.0 and o["nu"][0, 1, 1] == 1.0
    assert np.isinf(o["sigma2_c"][0, 0, 1])
    np.testing.assert_allclose(o["z"][0, :, 1], o["z_c"][0, 1, :, 1], rtol=1e-12)


# ----------------------------------------------------------------------------- fusion

def test_optimal_fusion_weights_properties():
    """Lemma 1: weights sum to one and minimize sum nu^2 sigma^2 on that simplex; Thm. 3 variance."""
    rng = np.random.default_rng(12)
    C, U, n = 5, 7, 3
    s2 = rng.uniform(0.1, 3.0, (C, U))
    zc = rng.standard_normal((C, U, n)) + 1j * rng.standard_normal((C, U, n))
    z, s2f, nu = lmmse.optimal_fusion(zc, s2)
    np.testing.assert_allclose(nu.sum(axis=0), 1.0, rtol=1e-14)
    assert (nu > 0).all()
    np.testing.assert_allclose(s2f, 1.0 / (1.0 / s2).sum(axis=0), rtol=1e-14)
    assert (s2f <= s2.min(axis=0)).all()
    fused_var = (nu ** 2 * s2).sum(axis=0)                    # variance of sum nu e_c (uncorrelated)
    np.testing.assert_allclose(fused_var, s2f, rtol=1e-12)   # the optimum equals Thm. 3
    for _ in range(200):                                      # no other point of the simplex is better
        d = rng.standard_normal((C, U))
        d -= d.mean(axis=0)
        other = nu + 0.05 * d
        assert ((other ** 2 * s2).sum(axis=0) >= fused_var - 1e-15).all()
    np.testing.assert_allclose(z, np.einsum("cu,cun->un", nu, zc), rtol=1e-14)


def test_fd_unbiased_fusion_is_unbiased_and_literal_is_not():
    """Unbiased local estimates fuse to an unbiased estimate (Lemma 1's model); literal ones keep the bias."""
    p = synth.make_problem(64, 16, 4, 300, 14, snr_db=0.0, seed=13)
    for est, lo, hi in (("unbiased", 0.98, 1.02), ("literal", 0.3, 0.95)):
        o = lmmse.equalize_fd(p.H, p.y, p.N0, p.Es, 4, est)
        g = np.real(np.mean(np.conj(p.s) * o["z"])) / p.Es
        assert lo < g < hi, (est, g)


# ----------------------------------------------------------------------------- large system

def _emp_sinr_db(o, p):
    return theory.db(p.Es / np.mean(np.abs(o["z"] - p.s) ** 2))


@pytest.mark.slow
@pytest.mark.parametrize("snr_db", [0.0, 6.0, 12.0, 20.0])
def test_large_system_sinr_matches_cor1_and_lemma5(snr_db):
    """B=256, U=16, C=8 Rayleigh: empirical unbiased SINR vs Cor. 1 (PD) and Lemma 5/7 (FD), FD <= PD.

    400 subcarriers x 14 symbols x 16 users = 89600 error samples per point;
    tolerance 0.25 dB (PD) and 0.5 dB (FD) covers finite-size bias and MC error.
    """
    B, U, C = 256, 16, 8
    p = synth.make_problem(B, U, C, 400, 14, snr_db=snr_db, seed=int(100 + snr_db))
    beta, a = U / B, B * p.Es / p.N0
    pd = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, C)
    fd = lmmse.equalize_fd(p.H, p.y, p.N0, p.Es, C)
    e_pd, e_fd = _emp_sinr_db(pd, p), _emp_sinr_db(fd, p)
    assert abs(e_pd - theory.db(theory.sinr_pd("lmmse", beta, a))) < 0.25
    assert abs(e_fd - theory.db(theory.sinr_fd_lmmse_uniform(beta, a, C))) < 0.5
    assert e_fd < e_pd                                                          # Lemma 3


@pytest.mark.slow
def test_nonuniform_clusters_match_lemma5():
    """Unequal clusters w = (3/4, 1/4): FD SINR follows Lemma 5; equal weights would lose ~1 dB here."""
    B, U = 128, 16
    p = synth.make_problem(B, U, 2, 400, 14, snr_db=10.0, seed=21)
    beta, a = U / B, B * p.Es / p.N0
    fd = lmmse.equalize_fd(p.H, p.y, p.N0, p.Es, 2, cluster_sizes=[96, 32])
    pred = theory.db(theory.sinr_fd_lmmse(beta, a, [0.75, 0.25]))
    assert abs(_emp_sinr_db(fd, p) - pred) < 0.5
    z_eq = 0.5 * (fd["z_c"][:, 0] + fd["z_c"][:, 1])                           # wrong (equal) weights
    e_eq = theory.db(p.Es / np.mean(np.abs(z_eq - p.s) ** 2))
    assert e_eq < pred - 0.8


# ----------------------------------------------------------------------------- theory

@pytest.mark.parametrize("kind", ["mrc", "zf", "lmmse"])
@pytest.mark.parametrize("beta", [0.0625, 0.25, 0.5])
@pytest.mark.parametrize("snr", [0.5, 10.0, 300.0])
def test_cor1_closed_forms_solve_the_tse_hanly_fixed_point(kind, beta, snr):
    """Cor. 1 equals Es / sigma^2 with sigma^2 the root of Thm. 1 (found by bisection)."""
    s2 = theory.fixed_point(kind, beta, 1.0 / snr, 1.0)
    assert theory.sinr_pd(kind, beta, snr) == pytest.approx(1.0 / s2, rel=1e-9)


def test_lemma5_is_the_sum_of_lemma2_cluster_sinrs():
    """Lemma 5 = sum_c Es/sigma_c^2 (Thm. 3) with sigma_c^2 from the per-cluster fixed point (Lemma 2)."""
    for beta, snr, w in ((0.0625, 40.0, [0.5, 0.3, 0.2]), (0.125, 3.0, [0.25] * 4), (0.2, 900.0, [0.9, 0.1])):
        tot = sum(1.0 / theory.fixed_point("lmmse", beta, 1.0 / snr, 1.0, wc) for wc in w)
        assert theory.sinr_fd_lmmse(beta, snr, w) == pytest.approx(tot, rel=1e-9)


def test_partition_lemmas_6_and_7():
    """Uniform clusters attain the Lemma 7 bound; all antennas in one cluster attain PD (Lemma 6); FD <= PD."""
    rng = np.random.default_rng(14)
    for beta, snr, C in ((0.0625, 160.0, 8), (0.1, 10.0, 4), (0.03, 1000.0, 16)):
        lo = theory.sinr_fd_lmmse_uniform(beta, snr, C)
        assert theory.sinr_fd_lmmse(beta, snr, [1.0 / C] * C) == pytest.approx(lo, rel=1e-12)
        pd = theory.sinr_pd("lmmse", beta, snr)
        assert theory.sinr_fd_lmmse(beta, snr, [1.0] + [0.0] * (C - 1)) == pytest.approx(pd, rel=1e-12)
        for _ in range(50):
            w = rng.dirichlet(np.ones(C))
            v = theory.sinr_fd_lmmse(beta, snr, w)
            assert lo - 1e-9 <= v <= pd + 1e-9


def test_lemma4_zf_fusion():
    """FD-ZF: sum of per-cluster ZF SINRs (w_c - beta) Es/N0 equals (Es/N0)(1 - C beta)."""
    beta, snr, w = 0.05, 30.0, [0.4, 0.35, 0.25]
    tot = sum(1.0 / theory.fixed_point("zf", beta, 1.0 / snr, 1.0, wc) for wc in w)
    assert theory.sinr_fd_zf(beta, snr, 3) == pytest.approx(tot, rel=1e-9)


def test_paper_message_sizes():
    """Sec. VI-C prints m_PD = 17.58 MB and m_FD = 8.20 MB (complex64, MiB) for U=16, C=4."""
    g = json.load(open(GOLDEN))["message_sizes"]
    m_pd, m_fd = theory.message_entries(g["U"], g["N_sc"], g["N_sym"], g["C"])
    mib = lambda e: e * g["bytes_per_entry"] / 2.0 ** 20
    assert round(mib(m_pd), 2) == g["m_PD_MiB"]
    assert round(mib(m_fd), 2) == g["m_FD_MiB"]
    assert round(2 * round(mib(m_fd), 2), 2) == g["m_CS_MiB"]   # the paper doubles the rounded m_FD


# ----------------------------------------------------------------------------- LLR

def test_qpsk_llr_closed_form():
    """QPSK max-log LLR is linear: -4 d Re(z) / sigma^2 (I bit), d = sqrt(Es/2)."""
    rng = np.random.default_rng(15)
    z = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    s2 = rng.uniform(0.1, 2.0, 50)
    Es = 1.7
    L = llr.maxlog_llr(z, s2, 2, Es)
    d = math.sqrt(Es / 2)
    np.testing.assert_allclose(L[:, 0], -4 * d * z.real / s2, rtol=1e-12)
    np.testing.assert_allclose(L[:, 1], -4 * d * z.imag / s2, rtol=1e-12)


@pytest.mark.parametrize("bits", [2, 4, 6])
def test_llr_signs_recover_labels_and_gray_property(bits):
    """At a constellation point the LLR signs give its label; neighbours differ in exactly one bit."""
    pts, labels = llr.qam_alphabet(bits, 1.0)
    L = llr.maxlog_llr(pts, 1e-3, bits, 1.0)
    assert np.array_equal((L < 0).astype(int), labels)
    M = len(pts)
    dmin = np.min(np.abs(pts[:, None] - pts[None, :]) + np.eye(M) * 1e9)
    for i in range(M):
        for j in range(M):
            if abs(abs(pts[i] - pts[j]) - dmin) < 1e-9:
                assert np.sum(labels[i] != labels[j]) == 1
    np.testing.assert_allclose(np.mean(np.abs(pts) ** 2), 1.0, rtol=1e-12)


def test_generator_levels_map_to_oracle_labels():
    """Noiseless, well-conditioned ZF: LLR hard decisions equal the labels of the drawn levels."""
    p = synth.make_problem(64, 4, 1, 10, 5, noiseless=True, seed=16, bits=4)
    o = lmmse.equalize_pd(p.H, p.y, 0.0, p.Es, 1)
    L = llr.maxlog_llr(o["z"], 1.0, 4, p.Es)
    assert np.array_equal((L < 0).astype(int), llr.hard_bits(p.levels, 4))
