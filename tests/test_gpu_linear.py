"""GPU parity of the ZF and MRC equalizers (Sec. III-A) in the PD and FD architectures.

The CUDA path (through the C ABI, ``ffeq_problem.equalizer``) against the FP64
oracle ``oracle.linear`` on the same seeded complex64 inputs.  Per subcarrier,
the relative 2-norm error of z, sigma^2 and the LLRs, and each entry's error
relative to max(|entry|, rms of the subcarrier) (``tests/parity.py``), must stay within
  * MRC: the tolerance of the local preprocessing's arithmetic (1e-5 FP32 and
    TF32x3, 2e-4 BF16x3, 2e-5 FP16x3); nothing is inverted;
  * ZF: max(that tolerance, 2 u kappa), kappa the largest condition number of the
    matrices inverted on that subcarrier (G, or every G_c for FD) and u the unit
    roundoff of the Gram arithmetic: without regularization the error of the
    preprocessing reaches the estimate amplified by kappa.
"""
import numpy as np
import pytest

import parity
from oracle import linear, lmmse
from oracle import llr as ollr
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC_TOL = {0: 1e-5, 1: 1e-5, 2: 2e-4, 3: 2e-5}      # FP32, TF32X3, BF16X3, FP16X3
UNIT = {0: 2.0 ** -22, 1: 2.0 ** -21, 2: 2.0 ** -16, 3: 2.0 ** -21}
EQ = {"zf": 1, "mrc": 2}


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


def _gpu(ff, p, arch, eq, llr_bits=0, precision=0, H=None, y=None, N0=None, **kw):
    dev = torch.device("cuda:0")
    Ht = torch.from_numpy(p.H if H is None else H).to(dev)
    yt = torch.from_numpy(p.y if y is None else y).to(dev)
    out = ff.equalize(Ht, yt, p.N0 if N0 is None else N0, p.Es, p.C, arch=arch, llr_bits=llr_bits,
                      with_info=True, precision=precision, equalizer=EQ[eq], **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle(p, arch, eq, idx=None, H=None, y=None, N0=None, sizes=None):
    H = p.H if H is None else H
    y = p.y if y is None else y
    if idx is not None:
        H, y = H[idx], y[idx]
    f = linear.equalize_pd_linear if arch == 0 else linear.equalize_fd_linear
    N0 = float(np.float32(p.N0)) if N0 is None else N0
    return f(H, y, N0, p.Es, p.C, eq, cluster_sizes=sizes)


def _kappa(p, arch, idx=None, sizes=None):
    """Largest cond_2 of the matrices ZF inverts, per subcarrier (G for PD, every G_c for FD)."""
    ks = range(p.n_sc) if idx is None else idx
    out = []
    for k in ks:
        Hm = p.H[k].astype(np.complex128).T
        bounds = [(0, p.B)] if arch == 0 else lmmse.partition(p.B, p.C, sizes)
        out.append(max(np.linalg.cond(Hm[b0:b1].conj().T @ Hm[b0:b1]) for b0, b1 in bounds))
    return np.array(out)


def _check(g, o, p, eq, arch, precision, bits=0, idx=None, sizes=None):
    z = g["z"] if idx is None else g["z"][idx]
    s2 = g["sigma2"] if idx is None else g["sigma2"][idx]
    tol = np.full(z.shape[0], PREC_TOL[precision])
    if eq == "zf":
        tol = np.maximum(tol, 2.0 * UNIT[precision] * _kappa(p, arch, idx, sizes))
    parity.check("z", z, o["z"], tol)
    parity.check("sigma2", s2, o["sigma2"], tol)
    if bits:
        L = g["llr"] if idx is None else g["llr"][idx]
        Lo = ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], bits, p.Es)
        parity.check("llr", L, Lo, 4 * tol)


CASES = [
    # B, U, C, n_sc, n_sym, bits, snr_db, Es
    (32, 4, 2, 64, 1, 2, 10.0, 1.0),        # small case (QPSK)
    (64, 16, 4, 37, 14, 4, 10.0, 1.0),      # several tiles, ragged subcarrier count, S = U (MRC only for FD)
    (48, 7, 3, 5, 3, 4, 5.0, 2.0),          # odd U, C = 3, Es != 1
    (256, 16, 8, 24, 14, 4, 20.0, 1.0),     # per-subcarrier shape of the throughput workload
    (256, 32, 16, 12, 14, 6, 15.0, 1.0),    # S = 16 < U = 32 (MRC only for FD)
    (33, 5, 3, 9, 2, 2, 8.0, 1.0),          # odd B: plain-load staging path
    (128, 1, 4, 10, 1, 2, 0.0, 1.0),        # single user
    (64, 32, 1, 10, 16, 8, 12.0, 1.0),      # U = 32, n_sym = 16 (maxima), C = 1
    (96, 12, 12, 6, 5, 6, 18.0, 1.0),       # C = 12, S = 8 < U (MRC only for FD)
]


@pytest.mark.parametrize("B,U,C,n_sc,n_sym,bits,snr,Es", CASES)
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("eq", ["zf", "mrc"])
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_parity_small(ff, B, U, C, n_sc, n_sym, bits, snr, Es, arch, eq, precision):
    if eq == "zf" and arch == 1 and B // C < U + 4:
        # S < U: G_c singular (ZF undefined); S = U: square Wishart G_c whose smallest
        # eigenvalue falls below the BF16x3 Gram error in about 1 of 60 draws.
        pytest.skip("ZF needs clusters with a few more antennas than users")
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=snr, bits=bits, seed=B * 131 + U * 7 + C, Es=Es)
    g = _gpu(ff, p, arch, eq, llr_bits=bits, precision=precision)
    o = _oracle(p, arch, eq)
    _check(g, o, p, eq, arch, precision, bits)
    assert (g["info"] == 0).all()


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("eq", ["zf", "mrc"])
@pytest.mark.parametrize("precision", [0, 2], ids=["fp32", "bf16x3"])
def test_full_size_throughput_workload_sampled(ff, arch, eq, precision):
    """B=256, U=16, C=8, 1200 subcarriers x 14 symbols, 16-QAM; 48 sampled subcarriers."""
    p = synth.make_problem(256, 16, 8, 1200, 14, snr_db=10.0, bits=4, seed=2024)
    g = _gpu(ff, p, arch, eq, llr_bits=4, precision=precision)
    idx = np.random.default_rng(5).choice(1200, 48, replace=False)
    _check(g, _oracle(p, arch, eq, idx=idx), p, eq, arch, precision, 4, idx=idx)
    assert np.isfinite(g["z"]).all() and np.isfinite(g["llr"]).all() and (g["info"] == 0).all()


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_noiseless_zf_recovers_the_symbols(ff, arch):
    p = synth.make_problem(128, 8, 4, 32, 6, noiseless=True, seed=4, bits=4)
    for precision in (0, 2):
        g = _gpu(ff, p, arch, "zf", precision=precision)
        assert np.abs(g["z"] - p.s).max() < (2e-3 if precision == 2 else 1e-4)
        assert (g["sigma2"] == 0).all()


def test_noiseless_single_user_mrc_takes_the_limit_weights(ff):
    """U = 1, N0 = 0: no interference, every variance 0, weights proportional to G_c,uu."""
    p = synth.make_problem(64, 1, 4, 16, 3, noiseless=True, seed=13, bits=2)
    for arch in (0, 1):
        g = _gpu(ff, p, arch, "mrc", N0=0.0)
        o = _oracle(p, arch, "mrc", N0=0.0)
        assert np.abs(g["z"] - p.s).max() < 1e-4
        parity.check("z", g["z"], o["z"], 1e-5)
        assert (g["sigma2"] == 0).all()


def test_singular_zf_reports_the_pivot_and_mrc_gives_zero_weight(ff):
    """User 2 invisible to cluster 0 on subcarrier 1: G_0 is singular there (ZF info = 3 and
    NaN outputs on that subcarrier); MRC gives that cluster weight 0 for the user."""
    p = synth.make_problem(32, 4, 2, 3, 2, seed=15)
    H = p.H.copy()
    H[1, 2, :16] = 0.0
    g = _gpu(ff, p, 1, "zf", H=H)
    assert g["info"].tolist() == [[0, 0], [3, 0], [0, 0]]
    assert np.isnan(g["z"][1]).all() and np.isfinite(g["z"][[0, 2]]).all()
    o = _oracle(p, 1, "zf", H=H)
    parity.check("z", g["z"][[0, 2]], o["z"][[0, 2]], 1e-4)
    g = _gpu(ff, p, 1, "mrc", H=H)
    o = _oracle(p, 1, "mrc", H=H)
    assert (g["info"] == 0).all()
    parity.check("z", g["z"], o["z"], 1e-5)
    parity.check("sigma2", g["sigma2"], o["sigma2"], 1e-5)


@pytest.mark.parametrize("eq", ["zf", "mrc"])
@pytest.mark.parametrize("precision", [0, 2], ids=["fp32", "bf16x3"])
def test_unequal_clusters(ff, eq, precision):
    sizes = [16, 48, 32, 24, 40, 32, 40, 24]
    p = synth.make_problem(256, 16, 8, 40, 14, snr_db=15.0, bits=4, seed=280)
    g = _gpu(ff, p, 1, eq, llr_bits=4, precision=precision, cluster_sizes=sizes)
    _check(g, _oracle(p, 1, eq, sizes=sizes), p, eq, 1, precision, 4, sizes=sizes)


@pytest.mark.parametrize("steps", [1, 2])
def test_zf_with_refinement(ff, steps):
    """ZF is the sweep with rho = 0, so the refinement from the inputs applies as for L-MMSE."""
    p = synth.make_problem(128, 16, 4, 20, 5, snr_db=20.0, bits=4, seed=8, corr_r=0.5)
    g = _gpu(ff, p, 1, "zf", precision=2, refine=steps)
    o = _oracle(p, 1, "zf")
    kap = _kappa(p, 1)
    tol = np.maximum(1e-5, 2.0 * 2.0 ** -22 * kap)
    if steps == 1:
        tol = np.maximum(tol, 4.0 * (2.0 ** -16 * kap) ** 2)
    parity.check("z", g["z"], o["z"], tol)


def test_mrc_zero_variance_takes_the_limit_weights(ff):
    """N0 = 0 with users of disjoint support (noisy inputs read as noiseless): user 0
    has no interference in clusters 0 and 1, so its variance there is exactly 0 and
    the N0 -> 0 limit of Lemma 1's weights applies (those clusters share the weight
    in proportion to G_c,uu; fused variance 0); users 1 and 2 keep the ordinary
    weights.  PD at C = 1 with two users on disjoint antennas is z = y^MRC_u / G_uu
    with variance 0.  Both against the oracle, element-wise."""
    p = synth.make_problem(64, 3, 4, 4, 2, snr_db=10.0, seed=18)
    n = p.y.astype(np.complex128) - p.s @ p.H.astype(np.complex128)
    H = p.H.copy()
    H[:, 1:, :32] = 0.0
    H[:, 0, 48:] = 0.0
    y = (p.s @ H.astype(np.complex128) + n).astype(np.complex64)
    for arch in (0, 1):
        for precision in (0, 2):
            g = _gpu(ff, p, arch, "mrc", H=H, y=y, N0=0.0, precision=precision)
            o = _oracle(p, arch, "mrc", H=H, y=y, N0=0.0)
            parity.check("z", g["z"], o["z"], PREC_TOL[precision])
            parity.check("sigma2", g["sigma2"], o["sigma2"], PREC_TOL[precision])
            assert np.array_equal(g["sigma2"] == 0, o["sigma2"] == 0)
            if arch == 1:
                assert (g["sigma2"][:, 0] == 0).all()
    q = synth.make_problem(32, 2, 1, 3, 2, snr_db=10.0, seed=19)
    n = q.y.astype(np.complex128) - q.s @ q.H.astype(np.complex128)
    H = q.H.copy()
    H[:, 0, 16:] = 0.0
    H[:, 1, :16] = 0.0
    y = (q.s @ H.astype(np.complex128) + n).astype(np.complex64)
    for arch in (0, 1):
        g = _gpu(ff, q, arch, "mrc", H=H, y=y, N0=0.0)
        o = _oracle(q, arch, "mrc", H=H, y=y, N0=0.0)
        parity.check("z", g["z"], o["z"], PREC_TOL[0])
        assert (g["sigma2"] == 0).all() and (o["sigma2"] == 0).all()
