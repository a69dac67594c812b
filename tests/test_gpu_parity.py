"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: per subcarrier, ||z_gpu - z_oracle||_2 / ||z_oracle||_2, and every
entry |z_gpu - z_oracle| / max(|z_oracle|, rms of the subcarrier's z_oracle)
(``tests/parity.py``), and the same for sigma^2 (and 4x for the LLRs, which are
affine in z with slope 2|a_0 - a_1| / sigma^2 and so carry the errors of both)
of that subcarrier, must not exceed max(t, 2 u kappa), kappa the largest
cond_2(G_c + rho I) of the matrices inverted on that subcarrier (G + rho I for
PD) and u the unit roundoff of the preprocessing (2^-22 FP32, 2^-21 TF32x3 and
FP16x3, 2^-16 BF16x3: the first-order bound of a solve whose matrix and
right-hand side carry relative errors u), with t
  * 1e-5 for the FP32 and TF32x3 local preprocessing (FP32-level arithmetic);
  * 2e-4 for BF16x3: a BF16 hi/lo pair carries 16 significand bits (relative
    error 2^-17 = 7.6e-6 per operand), and the solve amplifies the Gram error by
    kappa(G_c + rho I), which reaches about 250 in the S < U cases below;
  * 2e-5 for FP16x3: hi/lo pairs carry 22 bits like TF32x3, but the lo part of
    an entry below 2^-3 is an FP16 subnormal (absolute error up to 2^-25).
Inputs are the same seeded complex64 arrays for both sides.
"""
import numpy as np
import pytest

import parity
from oracle import llr as ollr
from oracle import lmmse
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
PREC_TOL = {0: 1e-5, 1: 1e-5, 2: 2e-4, 3: 2e-5}      # FP32, TF32X3, BF16X3, FP16X3


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


def _gpu(ff, p, arch, estimate, llr_bits=0, with_info=True, H=None, y=None, N0=None, precision=0):
    dev = torch.device("cuda:0")
    Ht = torch.from_numpy(p.H if H is None else H).to(dev)
    yt = torch.from_numpy(p.y if y is None else y).to(dev)
    out = ff.equalize(Ht, yt, p.N0 if N0 is None else N0, p.Es, p.C, arch=arch, estimate=estimate,
                      llr_bits=llr_bits, with_info=with_info, precision=precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle(p, arch, estimate, H=None, y=None, N0=None, idx=None):
    H = p.H if H is None else H
    y = p.y if y is None else y
    if idx is not None:
        H, y = H[idx], y[idx]
    f = lmmse.equalize_pd if arch == 0 else lmmse.equalize_fd
    return f(H, y, p.N0 if N0 is None else N0, p.Es, p.C, "unbiased" if estimate == 0 else "literal")


UNIT = {0: 2.0 ** -22, 1: 2.0 ** -21, 2: 2.0 ** -16, 3: 2.0 ** -21}


def _kappa(p, arch, idx=None, sizes=None):
    """Largest cond_2 of the regularized matrices inverted on each subcarrier:
    G + rho I (PD) or every G_c + rho I (FD)."""
    rho = float(np.float32(p.N0)) / p.Es
    ks = range(p.n_sc) if idx is None else idx
    parts = [(0, p.B)] if arch == 0 else lmmse.partition(p.B, p.C, sizes)
    out = []
    for k in ks:
        Hm = p.H[k].astype(np.complex128).T
        out.append(max(np.linalg.cond(Hm[b0:b1].conj().T @ Hm[b0:b1] + rho * np.eye(p.U)) for b0, b1 in parts))
    return np.array(out)


def _bound(p, arch, precision, idx=None):
    return np.maximum(PREC_TOL[precision], 2.0 * UNIT[precision] * _kappa(p, arch, idx))


def _check(g, o, p, bits=0, tol=TOL, idx=None):
    z = g["z"] if idx is None else g["z"][idx]
    s2 = g["sigma2"] if idx is None else g["sigma2"][idx]
    ez, _ = parity.check("z", z, o["z"], tol)
    parity.check("sigma2", s2, o["sigma2"], tol)
    if bits:
        L = g["llr"] if idx is None else g["llr"][idx]
        Lo = ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], bits, p.Es)
        parity.check("llr", L, Lo, 4 * tol)
    return ez


CASES = [
    # B, U, C, n_sc, n_sym, bits, snr_db, Es
    (32, 4, 2, 64, 1, 2, 10.0, 1.0),        # small PD/FD case (QPSK, 10 dB)
    (64, 16, 4, 37, 14, 4, 10.0, 1.0),      # several tiles, ragged subcarrier count
    (48, 7, 3, 5, 3, 4, 5.0, 2.0),          # odd U, C=3, Es != 1
    (256, 16, 8, 24, 14, 4, 20.0, 1.0),     # per-subcarrier shape of the throughput workload
    (256, 32, 16, 12, 14, 6, 15.0, 1.0),    # S=16 < U=32: rank-deficient local Gram matrices
    (33, 5, 3, 9, 2, 2, 8.0, 1.0),          # odd B: plain-load staging path
    (128, 1, 4, 10, 1, 2, 0.0, 1.0),        # single user
    (64, 32, 1, 10, 16, 8, 12.0, 1.0),      # U=32, n_sym=16 (maxima), C=1, 256-QAM LLRs
    (40, 20, 5, 7, 4, 4, 6.0, 0.5),         # S=8 < U=20, C=5 (split-K with 3 spare warps)
    (96, 12, 12, 6, 5, 6, 18.0, 1.0),       # C=12: two rounds of clusters
]


@pytest.mark.parametrize("B,U,C,n_sc,n_sym,bits,snr,Es", CASES)
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("estimate", [0, 1], ids=["unbiased", "literal"])
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_parity_small(ff, B, U, C, n_sc, n_sym, bits, snr, Es, arch, estimate, precision):
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=snr, bits=bits, seed=B * 131 + U * 7 + C, Es=Es)
    g = _gpu(ff, p, arch, estimate, llr_bits=bits, precision=precision)
    o = _oracle(p, arch, estimate)
    _check(g, o, p, bits, tol=_bound(p, arch, precision))
    assert (g["info"] == 0).all()


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_parity_correlated_channel(ff, arch, precision):
    """Receive-side exponential correlation r = 0.7 (ill-conditioned local Gram matrices)."""
    p = synth.make_problem(256, 32, 16, 8, 14, snr_db=15.0, bits=6, seed=77, corr_r=0.7)
    g = _gpu(ff, p, arch, 0, llr_bits=6, precision=precision)
    o = _oracle(p, arch, 0)
    _check(g, o, p, 6, tol=_bound(p, arch, precision))


def test_pd_ignores_partition_and_equals_fd_at_c1(ff):
    p = synth.make_problem(64, 8, 1, 16, 3, seed=3)
    base = _gpu(ff, p, 0, 0)
    for C in (2, 4, 8, 16):
        q = synth.make_problem(64, 8, C, 16, 3, seed=3)
        g = _gpu(ff, q, 0, 0)
        assert np.array_equal(g["z"], base["z"]) and np.array_equal(g["sigma2"], base["sigma2"])
    fd = _gpu(ff, p, 1, 0)
    assert np.array_equal(fd["z"], base["z"]) and np.array_equal(fd["sigma2"], base["sigma2"])


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_noiseless_zero_forcing(ff, arch, precision):
    p = synth.make_problem(128, 8, 4, 32, 6, noiseless=True, seed=4, bits=4)
    g = _gpu(ff, p, arch, 0, precision=precision)
    assert np.abs(g["z"] - p.s).max() < (2e-3 if precision == 2 else 1e-4)
    assert (g["sigma2"] == 0).all()


def test_singular_zero_forcing_reports_pivot(ff):
    p = synth.make_problem(16, 4, 2, 3, 2, noiseless=True, seed=10)
    H = p.H.copy()
    H[1, 2, :] = 0.0
    for arch in (0, 1):
        g = _gpu(ff, p, arch, 0, H=H, N0=0.0)
        o = _oracle(p, arch, 0, H=H, N0=0.0)
        assert np.array_equal(g["info"].reshape(o["info"].shape), o["info"])
        assert np.isnan(g["z"][1]).all() and np.isnan(g["sigma2"][1]).all()
        assert np.isfinite(g["z"][[0, 2]]).all()


def test_zero_channel_column_gets_zero_weight(ff):
    p = synth.make_problem(16, 3, 2, 2, 2, seed=11)
    H = p.H.copy()
    H[0, 1, :8] = 0.0            # invisible to cluster 0 only: FD weight 0 there
    H[1, 2, :] = 0.0             # invisible everywhere: z = 0, sigma^2 = inf
    for arch in (0, 1):
        g = _gpu(ff, p, arch, 0, H=H)
        o = _oracle(p, arch, 0, H=H)
        assert np.isinf(g["sigma2"][1, 2]) and np.isinf(o["sigma2"][1, 2])
        assert (g["z"][1, :, 2] == 0).all()
        keep = np.ones_like(o["sigma2"], bool)
        keep[1, 2] = False
        np.testing.assert_allclose(g["sigma2"][keep], o["sigma2"][keep], rtol=TOL)
        np.testing.assert_allclose(g["z"][0], o["z"][0], rtol=TOL, atol=TOL)


def test_empty_and_single_subcarrier(ff):
    p = synth.make_problem(32, 4, 2, 1, 1, seed=12)
    for arch in (0, 1):
        _check(_gpu(ff, p, arch, 0), _oracle(p, arch, 0), p)
    dev = torch.device("cuda:0")
    plan = ff.ffeq_plan_create(32, 4, 2, 0, 1)
    ff.ffeq_equalize(plan, None, None, 1.0, 1.0, None, None)


def test_host_buffer_entry_point_matches_device_path(ff):
    p = synth.make_problem(64, 16, 4, 40, 14, seed=13, bits=4)
    plan = ff.ffeq_plan_create(64, 16, 4, 40, 14, arch=ff.FD, llr_bits=4)
    nbytes = ff.ffeq_host_staging_size(plan)
    staging = torch.empty(nbytes, dtype=torch.uint8, device="cuda:0")
    Hh = torch.from_numpy(p.H).pin_memory()
    yh = torch.from_numpy(p.y).pin_memory()
    z = torch.empty((40, 14, 16), dtype=torch.complex64).pin_memory()
    s2 = torch.empty((40, 16), dtype=torch.float32).pin_memory()
    L = torch.empty((40, 14, 16, 4), dtype=torch.float32).pin_memory()
    info = torch.empty((40, 4), dtype=torch.int32).pin_memory()
    ff.ffeq_equalize_host(plan, Hh, yh, p.N0, p.Es, z, s2, L, info, staging, nbytes)
    g = _gpu(ff, p, 1, 0, llr_bits=4)
    assert np.array_equal(z.numpy(), g["z"]) and np.array_equal(s2.numpy(), g["sigma2"])
    assert np.array_equal(L.numpy(), g["llr"]) and (info.numpy() == 0).all()
    assert ff.ffeq_device_status() == 0


@pytest.mark.parametrize("pinned", [True, False], ids=["in-place", "staged"])
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_host_entry_point_both_paths(ff, arch, pinned):
    """Page-locked buffers are read and written in place by the kernels; pageable
    ones go through the staging copies.  Both equal the device path bit for bit
    (inputs read over the host link take the plain-load contraction, shape 1:
    the device path is pinned to the same shape for that comparison)."""
    p = synth.make_problem(128, 12, 4, 33, 5, seed=17, bits=4)
    plan = ff.ffeq_plan_create(128, 12, 4, 33, 5, arch=arch, precision=ff.BF16X3, llr_bits=4)
    nbytes = ff.ffeq_host_staging_size(plan)
    staging = torch.empty(nbytes, dtype=torch.uint8, device="cuda:0")
    Ceff = 4 if arch == 1 else 1

    def buf(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.pin_memory() if pinned else t
    Hh, yh = buf(p.H), buf(p.y)
    z = buf(np.zeros((33, 5, 12), np.complex64))
    s2 = buf(np.zeros((33, 12), np.float32))
    L = buf(np.zeros((33, 5, 12, 4), np.float32))
    info = buf(np.full((33, Ceff), -1, np.int32))
    ff.ffeq_equalize_host(plan, Hh, yh, p.N0, p.Es, z, s2, L, info, staging, nbytes)
    if pinned:
        dplan = ff.ffeq_plan_create(128, 12, 4, 33, 5, arch=arch, precision=ff.BF16X3, llr_bits=4)
        ff.ffeq_plan_set_tuning(dplan, (1, 0))
        dev = torch.device("cuda:0")
        gz = torch.empty((33, 5, 12), dtype=torch.complex64, device=dev)
        gs = torch.empty((33, 12), dtype=torch.float32, device=dev)
        gl = torch.empty((33, 5, 12, 4), dtype=torch.float32, device=dev)
        nb = ff.ffeq_workspace_size(dplan)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        ff.ffeq_equalize(dplan, torch.from_numpy(p.H).to(dev), torch.from_numpy(p.y).to(dev), p.N0, p.Es, gz, gs, gl,
                         None, ws, nb)
        torch.cuda.synchronize()
        g = {"z": gz.cpu().numpy(), "sigma2": gs.cpu().numpy(), "llr": gl.cpu().numpy()}
    else:
        g = _gpu(ff, p, arch, 0, llr_bits=4, precision=2)
    assert np.array_equal(z.numpy(), g["z"]) and np.array_equal(s2.numpy(), g["sigma2"])
    assert np.array_equal(L.numpy(), g["llr"]) and (info.numpy() == 0).all()


@pytest.mark.parametrize("snr", [float(v) for v in range(0, 22, 2)])
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [0, 2], ids=["fp32", "bf16x3"])
def test_snr_sweep_of_the_throughput_shape(ff, snr, arch, precision):
    """The per-subcarrier shape of the throughput workload (B=256, U=16, C=8, 14
    symbols, 16-QAM) over its SNR sweep, 0..20 dB in 2 dB steps, FP32 and BF16x3
    contractions: every subcarrier of 96 against the oracle, z, sigma^2 and LLRs,
    within the precision's bound (kappa-aware)."""
    p = synth.make_problem(256, 16, 8, 96, 14, snr_db=snr, bits=4, seed=4000 + int(snr))
    g = _gpu(ff, p, arch, 0, llr_bits=4, precision=precision)
    _check(g, _oracle(p, arch, 0), p, 4, tol=_bound(p, arch, precision))
    assert (g["info"] == 0).all()


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_full_size_throughput_workload_sampled(ff, arch, precision):
    """B=256, U=16, C=8, 1200 subcarriers x 14 symbols, 16-QAM, in the benchmark's launch.

    The oracle checks 48 sampled subcarriers; every output must be finite."""
    p = synth.make_problem(256, 16, 8, 1200, 14, snr_db=10.0, bits=4, seed=2024)
    g = _gpu(ff, p, arch, 0, llr_bits=4, precision=precision)
    idx = np.random.default_rng(5).choice(1200, 48, replace=False)
    o = _oracle(p, arch, 0, idx=idx)
    _check(g, o, p, 4, tol=_bound(p, arch, precision, idx), idx=idx)
    assert np.isfinite(g["z"]).all() and np.isfinite(g["llr"]).all() and (g["info"] == 0).all()


def test_full_size_correlated_workload_sampled(ff):
    """B=256, U=32, C=16, 3300 x 14, 64-QAM, r=0.7, 15 dB (FD and PD), sampled."""
    p = synth.make_problem(256, 32, 16, 3300, 14, snr_db=15.0, bits=6, seed=7, corr_r=0.7)
    idx = np.random.default_rng(6).choice(3300, 24, replace=False)
    for arch in (0, 1):
        for precision in (0, 2):
            g = _gpu(ff, p, arch, 0, llr_bits=6, precision=precision)
            _check(g, _oracle(p, arch, 0, idx=idx), p, 6, tol=_bound(p, arch, precision, idx), idx=idx)
            assert np.isfinite(g["z"]).all()


def _kappa_clusters(p, sizes):
    """Largest cond_2(G_c + rho I) over the clusters of each subcarrier (FD)."""
    rho = float(np.float32(p.N0)) / p.Es
    out = np.ones(p.n_sc)
    for k in range(p.n_sc):
        Hm = p.H[k].astype(np.complex128).T
        for b0, b1 in lmmse.partition(p.B, p.C, sizes):
            Hc = Hm[b0:b1]
            out[k] = max(out[k], np.linalg.cond(Hc.conj().T @ Hc + rho * np.eye(p.U)))
    return out


CLUSTER_CASES = [  # B, U, C, n_sc, n_sym, sizes
    (100, 8, 3, 24, 3, [40, 35, 25]),                          # B % C != 0
    (256, 16, 8, 40, 14, [16, 48, 32, 24, 40, 32, 40, 24]),     # the throughput shape, unequal
    (128, 8, 3, 12, 2, [64, 0, 64]),                            # an empty cluster: its users get weight 0
    (96, 12, 5, 10, 5, [7, 33, 20, 30, 6]),                     # odd sizes and offsets, S < U
]


@pytest.mark.parametrize("case", CLUSTER_CASES)
@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp32", "tf32x3", "bf16x3", "fp16x3"])
def test_unequal_clusters_match_the_oracle(ff, case, precision):
    """Clusters of given sizes B_c (Sec. II-B) through ffeq_plan_create_clusters:
    FD against the oracle's partition with the same sizes (bound max(tolerance,
    2 u kappa) per subcarrier, kappa the largest local condition number), and PD,
    which sums every cluster, equal to the uniform-plan result."""
    B, U, C, n_sc, n_sym, sizes = case
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=15.0, bits=4, seed=B + U + C)
    dev = torch.device("cuda:0")
    H, y = torch.from_numpy(p.H).to(dev), torch.from_numpy(p.y).to(dev)
    g = ff.equalize(H, y, p.N0, p.Es, C, arch=1, llr_bits=4, with_info=True, precision=precision,
                    cluster_sizes=sizes)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    o = lmmse.equalize_fd(p.H, p.y, float(np.float32(p.N0)), p.Es, C, "unbiased", cluster_sizes=sizes)
    assert np.array_equal(g["info"], o["info"])
    tol = np.maximum(PREC_TOL[precision], 2.0 * UNIT[precision] * _kappa_clusters(p, sizes))
    parity.check("z", g["z"], o["z"], tol)
    parity.check("sigma2", g["sigma2"], o["sigma2"], tol)
    Lo = ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], 4, p.Es)
    parity.check("llr", g["llr"], Lo, 4 * tol)
    if B % C == 0:
        pd_sizes = ff.equalize(H, y, p.N0, p.Es, C, arch=0, precision=precision, cluster_sizes=sizes)
        pd_equal = ff.equalize(H, y, p.N0, p.Es, C, arch=0, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(pd_sizes["z"], pd_equal["z"]) and torch.equal(pd_sizes["sigma2"], pd_equal["sigma2"])


@pytest.mark.parametrize("steps", [1, 2])
def test_unequal_clusters_with_refinement(ff, steps):
    """Refinement re-reads each cluster's own antennas (offsets, not B / C)."""
    B, U, C, n_sc, n_sym, sizes = 96, 12, 5, 10, 5, [7, 33, 20, 30, 6]
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=20.0, bits=4, seed=7, corr_r=0.5)
    dev = torch.device("cuda:0")
    g = ff.equalize(torch.from_numpy(p.H).to(dev), torch.from_numpy(p.y).to(dev), p.N0, p.Es, C, arch=1,
                    with_info=True, precision=2, refine=steps, cluster_sizes=sizes)
    torch.cuda.synchronize()
    o = lmmse.equalize_fd(p.H, p.y, float(np.float32(p.N0)), p.Es, C, "unbiased", cluster_sizes=sizes)
    kap = _kappa_clusters(p, sizes)
    tol = np.maximum(1e-5, 2.0 * 2.0 ** -22 * kap)
    if steps == 1:
        tol = np.maximum(tol, 4.0 * (2.0 ** -16 * kap) ** 2)
    parity.check("z", g["z"].cpu().numpy(), o["z"], tol)
