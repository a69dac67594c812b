"""GPU parity of LAMA-PD and LAMA-FD (Sec. III-B, Algorithm 1) against the FP64 oracle.

The CUDA path (through the C ABI, ``ffeq_problem.equalizer = FFEQ_LAMA``) and
``oracle.lama`` on the same seeded complex64 inputs.  Per subcarrier, the
relative 2-norm error of z, of sigma^2 (one value per received vector) and of
the LLRs (4x), and each entry's error relative to max(|entry|, rms of the
subcarrier) (``tests/parity.py``), must stay within 2e-5 for the FP32 and TF32x3 preprocessing,
5e-5 for FP16x3 and 3e-4 for BF16x3.  No matrix is inverted; the posterior-mean
denoiser can amplify an input error by up to Var(s | z) / (tau / 2) per
iteration on symbols near a decision boundary, but on these cases (every
cluster at beta_c = U / S_c <= 1/2) perturbing the oracle's inputs by a
relative 1e-6 (1.5e-5) moves z by at most 2.2e-6 (1.9e-5): the bounds keep a
factor of 10 or more above that.
"""
import numpy as np
import pytest

import parity
from oracle import lama
from oracle import llr as ollr
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 2e-5, 1: 2e-5, 2: 3e-4, 3: 5e-5}


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


def _gpu(ff, p, arch, T, bits, precision=0, sizes=None):
    dev = torch.device("cuda:0")
    out = ff.equalize(torch.from_numpy(p.H).to(dev), torch.from_numpy(p.y).to(dev), p.N0, p.Es, p.C, arch=arch,
                      llr_bits=bits, with_info=True, precision=precision, equalizer=ff.LAMA, lama_iters=T,
                      cluster_sizes=sizes)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle(p, arch, T, bits, idx=None, sizes=None):
    H, y = (p.H, p.y) if idx is None else (p.H[idx], p.y[idx])
    f = lama.equalize_pd_lama if arch == 0 else lama.equalize_fd_lama
    return f(H, y, float(np.float32(p.N0)), p.Es, p.C, bits, T, cluster_sizes=sizes)


def _check(g, o, p, bits, tol, idx=None):
    z = g["z"] if idx is None else g["z"][idx]
    s2 = g["sigma2"] if idx is None else g["sigma2"][idx]
    parity.check("z", z, o["z"], tol)
    parity.check("sigma2", s2, o["sigma2"], tol)
    L = g["llr"] if idx is None else g["llr"][idx]
    Lo = ollr.maxlog_llr(o["z"], o["sigma2"], bits, p.Es)
    parity.check("llr", L, Lo, 4 * tol)


CASES = [
    # B, U, C, n_sc, n_sym, bits, snr_db, Es
    (32, 4, 2, 40, 1, 2, 10.0, 1.0),        # small case (QPSK)
    (128, 16, 4, 37, 14, 4, 12.0, 1.0),     # several CTAs per subcarrier, ragged subcarrier count
    (96, 7, 3, 5, 3, 4, 8.0, 2.0),          # odd U, C = 3, Es != 1
    (256, 16, 8, 24, 14, 4, 10.0, 1.0),     # per-subcarrier shape of the throughput workload
    (33, 5, 3, 9, 2, 2, 8.0, 1.0),          # odd B: plain-load staging path, S = 11
    (128, 1, 4, 10, 1, 2, 0.0, 1.0),        # single user
    (256, 32, 4, 6, 16, 6, 20.0, 1.0),      # U = 32, n_sym = 16 (maxima), 64-QAM
    (64, 8, 1, 10, 5, 8, 25.0, 1.0),        # C = 1, 256-QAM
]


@pytest.mark.parametrize("B,U,C,n_sc,n_sym,bits,snr,Es", CASES)
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_parity_small(ff, B, U, C, n_sc, n_sym, bits, snr, Es, arch, precision):
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=snr, bits=bits, seed=B * 17 + U * 3 + C, Es=Es)
    g = _gpu(ff, p, arch, 6, bits, precision)
    _check(g, _oracle(p, arch, 6, bits), p, bits, TOL[precision])
    assert (g["info"] == 0).all()


@pytest.mark.parametrize("T", [1, 2, 20])
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_iteration_counts(ff, T, arch):
    """T = 1 is the normalized matched filter; 20 iterations run past convergence."""
    p = synth.make_problem(128, 16, 4, 20, 6, snr_db=10.0, bits=4, seed=T)
    _check(_gpu(ff, p, arch, T, 4), _oracle(p, arch, T, 4), p, 4, TOL[0])


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [0, 2], ids=["fp32", "bf16x3"])
def test_full_size_throughput_workload_sampled(ff, arch, precision):
    """B=256, U=16, C=8, 1200 subcarriers x 14 symbols, 16-QAM, 10 dB, T = 8; 24 sampled subcarriers."""
    p = synth.make_problem(256, 16, 8, 1200, 14, snr_db=10.0, bits=4, seed=2024)
    g = _gpu(ff, p, arch, 8, 4, precision)
    idx = np.random.default_rng(5).choice(1200, 24, replace=False)
    _check(g, _oracle(p, arch, 8, 4, idx=idx), p, 4, TOL[precision], idx=idx)
    assert np.isfinite(g["z"]).all() and np.isfinite(g["llr"]).all()


def test_unequal_clusters_and_an_empty_one(ff):
    """Clusters of 64, 0 and 64 antennas: each runs in its own normalization; the empty one
    gets weight 0 (Lemma 1)."""
    sizes = [64, 0, 64]
    p = synth.make_problem(128, 8, 3, 12, 4, snr_db=10.0, bits=4, seed=9)
    g = _gpu(ff, p, 1, 6, 4, sizes=sizes)
    _check(g, _oracle(p, 1, 6, 4, sizes=sizes), p, 4, TOL[0])


def test_high_snr_hard_decisions_are_the_symbols(ff):
    p = synth.make_problem(128, 16, 2, 16, 8, snr_db=25.0, bits=4, seed=45)
    pts = lama.qam_points(4, p.Es)
    for arch in (0, 1):
        g = _gpu(ff, p, arch, 8, 4)
        hard = pts[np.argmin(np.abs(g["z"][..., None].astype(np.complex128) - pts), axis=-1)]
        assert np.abs(hard - p.s).max() < 1e-5
