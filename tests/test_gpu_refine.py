"""GPU parity of iterative refinement from the inputs (ffeq_problem.refine).

On ill-conditioned systems (receive correlation r = 0.7 across the array and
clusters with S = B/C not above U, high SNR) the mixed-precision preprocessing
is off by about kappa(G_c + rho I) * 2^-16; one or two refinement steps from H
and y must bring z and sigma^2 to the FP32-level bound max(1e-5, 2 kappa 2^-22)
per subcarrier (kappa the subcarrier's largest cond_2(G_c + rho I), as in the
batch tests), and at least 4x below the unrefined error where that exceeds
1e-5.  Refinement must not degrade well-conditioned problems.
"""
import numpy as np
import pytest

from oracle import llr as ollr
from oracle import lmmse
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-30)


def _kappa(p, arch):
    rho = float(np.float32(p.N0)) / p.Es
    parts = lmmse.partition(p.B, p.C) if arch == 1 else [(0, p.B)]
    out = np.ones(p.n_sc)
    for k in range(p.n_sc):
        Hm = p.H[k].astype(np.complex128).T
        for (b0, b1) in parts:
            Hc = Hm[b0:b1]
            out[k] = max(out[k], np.linalg.cond(Hc.conj().T @ Hc + rho * np.eye(p.U)))
    return out


def _run(ff, p, arch, precision, refine, bits=4, estimate=0):
    dev = torch.device("cuda:0")
    g = ff.equalize(torch.from_numpy(p.H).to(dev), torch.from_numpy(p.y).to(dev), p.N0, p.Es, p.C, arch=arch,
                    estimate=estimate, llr_bits=bits, with_info=True, precision=precision, refine=refine)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in g.items()}


CASES = [  # B, U, C, n_sc, n_sym, snr_db, corr_r
    (128, 16, 8, 24, 6, 30.0, 0.7),      # FD clusters S = U = 16, correlated
    (96, 12, 12, 16, 4, 25.0, 0.7),      # S = 8 < U
    (256, 32, 16, 8, 14, 30.0, 0.7),     # U = 32, S = 16 < U
    (64, 16, 2, 20, 3, 35.0, 0.8),       # PD-interesting: B/U = 4, strong correlation
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [2, 1], ids=["bf16x3", "tf32x3"])
def test_refinement_reaches_fp32_level(ff, case, arch, precision):
    B, U, C, n_sc, n_sym, snr, r = case
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=snr, bits=4, seed=B + U + C, corr_r=r)
    f = lmmse.equalize_pd if arch == 0 else lmmse.equalize_fd
    o = f(p.H, p.y, float(np.float32(p.N0)), p.Es, C, "unbiased")
    kap = _kappa(p, arch)
    bound = np.maximum(1e-5, 2.0 * 2.0 ** -22 * kap)
    base = _run(ff, p, arch, precision, 0)
    e0 = _rel(base["z"], o["z"])
    for steps in (1, 2):
        g = _run(ff, p, arch, precision, steps)
        assert (g["info"] == 0).all()
        ez, es = _rel(g["z"], o["z"]), _rel(g["sigma2"], o["sigma2"])
        need = bound if steps == 2 else np.maximum(bound, 4.0 * 2.0 ** -16 * kap * 2.0 ** -16 * kap)
        assert (ez <= need).all(), (steps, ez.max(), need[np.argmax(ez - need)], kap.max())
        assert (es <= need).all(), (steps, es.max(), kap.max())
        big = e0 > 1e-5
        if steps == 2 and big.any():
            assert (ez[big] <= e0[big] / 4).all(), (ez[big].max(), e0[big].max())
        Lo = ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], 4, p.Es)
        assert (_rel(g["llr"], Lo) <= 4 * need).all()


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_refinement_keeps_well_conditioned_results(ff, arch):
    p = synth.make_problem(256, 16, 8, 64, 14, snr_db=10.0, bits=4, seed=5)
    f = lmmse.equalize_pd if arch == 0 else lmmse.equalize_fd
    for estimate, est in ((0, "unbiased"), (1, "literal")):
        o = f(p.H, p.y, float(np.float32(p.N0)), p.Es, p.C, est)
        for precision in (0, 2):
            g = _run(ff, p, arch, precision, 1, estimate=estimate)
            assert _rel(g["z"], o["z"]).max() <= 1e-5, (precision, estimate)
            assert _rel(g["sigma2"], o["sigma2"]).max() <= 1e-5, (precision, estimate)


def test_refinement_reports_singular_systems(ff):
    p = synth.make_problem(16, 4, 2, 3, 2, noiseless=True, seed=10)
    H = p.H.copy()
    H[1, 2, :] = 0.0
    dev = torch.device("cuda:0")
    for arch in (0, 1):
        g = ff.equalize(torch.from_numpy(H).to(dev), torch.from_numpy(p.y).to(dev), 0.0, p.Es, p.C, arch=arch,
                        with_info=True, refine=1)
        torch.cuda.synchronize()
        o = (lmmse.equalize_pd if arch == 0 else lmmse.equalize_fd)(H, p.y, 0.0, p.Es, p.C, "unbiased")
        assert np.array_equal(g["info"].cpu().numpy().reshape(o["info"].shape), o["info"])
        assert np.isnan(g["z"][1].cpu().numpy()).all()
        assert np.isfinite(g["z"][[0, 2]].cpu().numpy()).all()
