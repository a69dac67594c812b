"""GPU parity of uneven batches (include/ffeq_batch.h) against the FP64 oracle.

Every instance of a batch is checked on its own against ``oracle.lmmse``
(``equalize_pd`` / ``equalize_fd`` on that instance's arrays) with the bounds of
the uniform parity tests: per subcarrier, relative 2-norm error of z, sigma^2
and the LLRs at most 1e-5 (FP32, TF32x3) or 2e-4 (BF16x3).  The uneven workload
is 4096 instances with U uniform on 4..32, B in {64, 128, 256}, C in
{1, 2, 4, 8, 16} (dividing B, at least 4 antennas per cluster), 1..14 OFDM
symbols, SNR uniform on 5..20 dB, 16-QAM.  Launch shapes (pipeline depth, solve
CTA width) must not change a single bit of the results (lanes per row change
the solve's rounding order only), and a CUDA-graph replay must equal the eager
call.

Random uneven instances include ill-conditioned ones (FD with S = B/C < U:
rank-deficient local Gram matrices, kappa(G_c + rho I) ~ lambda_max / rho in
the hundreds), so each instance's bound is
    max(flat bound, 2 u kappa),   kappa = max over its systems of cond_2(G_c + rho I),
the first-order perturbation bound of a linear solve whose matrix and
right-hand side carry relative errors u from the products that formed them:
u = 2^-16 for BF16x3 (hi + lo pairs keep 16 significand bits; the dropped lo*lo
term is 2^-18), 2^-21 for TF32x3 and FP16x3 (22 bits, dropped term 2^-22; FP16's
subnormal lo parts of entries below 2^-3 add at most 2^-25 absolute) and 2^-22
for FP32 (2^-24 per product, summation over up to 256 antennas).

The LLR bound is 4x the z bound.  Per bit the max-log LLR is affine in z with
slope 2 |a_0 - a_1| / sigma^2 (a_0, a_1 the nearest levels with the bit 0 / 1),
so its absolute error follows that of z, while its norm drops for symbols that
sit near a decision threshold; among thousands of random instances a few have
such subcarriers (worst seen: 1.04x the z bound, TF32x3, FD).
"""
import numpy as np
import pytest

import parity
from oracle import lama as olama
from oracle import linear as olinear
from oracle import llr as ollr
from oracle import lmmse
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC_TOL = {0: 1e-5, 1: 1e-5, 2: 2e-4, 3: 2e-5}      # FP32, TF32X3, BF16X3, FP16X3
UNIT = {0: 2.0 ** -22, 1: 2.0 ** -21, 2: 2.0 ** -16, 3: 2.0 ** -21}


def _kappa(p, arch):
    """Largest 2-norm condition number of the instance's systems (FP64)."""
    rho = float(np.float32(p.N0)) / p.Es
    parts = lmmse.partition(p.B, p.C) if arch == 1 else [(0, p.B)]
    worst = 1.0
    for k in range(p.n_sc):
        Hm = p.H[k].astype(np.complex128).T
        for (b0, b1) in parts:
            Hc = Hm[b0:b1]
            worst = max(worst, np.linalg.cond(Hc.conj().T @ Hc + rho * np.eye(p.U)))
    return worst


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


@pytest.fixture(scope="module")
def uneven():
    return synth.make_uneven(4096, seed=4)


def _specs(ps):
    return [(p.B, p.U, p.C, p.n_sc, p.n_sym, p.N0, p.Es) for p in ps]


class Run:
    """Device buffers of one packed batch and its plan."""

    def __init__(self, ff, ps, arch, precision=0, estimate=0, llr_bits=4, with_info=True, specs=None, equalizer=0,
                 lama_iters=0):
        dev = torch.device("cuda:0")
        self.ff, self.ps, self.arch, self.bits = ff, ps, arch, llr_bits
        cfg, inst = ff.pack_batch(specs or _specs(ps), arch=arch, precision=precision, estimate=estimate,
                                  llr_bits=llr_bits, with_info=with_info, equalizer=equalizer, lama_iters=lama_iters)
        self.cfg, self.inst = cfg, inst
        H, y = _flat(ps, cfg, inst)
        self.H = torch.from_numpy(H).to(dev)
        self.y = torch.from_numpy(y).to(dev)
        self.z = torch.full((max(1, cfg.z_elems),), complex("nan"), dtype=torch.complex64, device=dev)
        self.s2 = torch.full((max(1, cfg.sigma2_elems),), float("nan"), dtype=torch.float32, device=dev)
        self.llr = torch.full((max(1, cfg.llr_elems),), float("nan"), dtype=torch.float32, device=dev)
        self.info = torch.full((max(1, cfg.info_elems),), -1, dtype=torch.int32, device=dev)
        self.batch = ff.ffeq_batch_create(cfg, inst)
        self.nb = ff.ffeq_batch_workspace_size(self.batch)
        self.ws = torch.empty(max(self.nb, 256), dtype=torch.uint8, device=dev)

    def args(self):
        return (self.H, self.y, self.z, self.s2, self.llr if self.bits else None,
                self.info if self.cfg.info_elems else None, self.ws, self.nb)

    def equalize(self, stream=None):
        self.ff.ffeq_batch_equalize(self.batch, *self.args(), stream=stream)

    def host(self):
        torch.cuda.synchronize()
        return dict(z=self.z.cpu().numpy(), s2=self.s2.cpu().numpy(), llr=self.llr.cpu().numpy(),
                    info=self.info.cpu().numpy())


def _flat(ps, cfg, inst):
    H = np.zeros(cfg.h_elems, np.complex64)
    y = np.zeros(cfg.y_elems, np.complex64)
    for p, it in zip(ps, inst):
        H[it.h_off:it.h_off + p.H.size] = p.H.ravel()
        y[it.y_off:it.y_off + p.y.size] = p.y.ravel()
    return H, y


def _check(run, out, estimate=0, precision=0, skip=()):
    worst = 0.0
    for idx, (p, it) in enumerate(zip(run.ps, run.inst)):
        if idx in skip or p.n_sc == 0:
            continue
        tol = max(PREC_TOL[precision], 2.0 * UNIT[precision] * _kappa(p, run.arch))
        f = lmmse.equalize_pd if run.arch == 0 else lmmse.equalize_fd
        o = f(p.H, p.y, float(np.float32(p.N0)), p.Es, p.C, "unbiased" if estimate == 0 else "literal")
        n, U, NS = p.n_sc, p.U, p.n_sym
        z = out["z"][it.z_off:it.z_off + n * NS * U].reshape(n, NS, U)
        s2 = out["s2"][it.sigma2_off:it.sigma2_off + n * U].reshape(n, U)
        ez, _ = parity.check(f"z[{idx}]", z, o["z"], tol)
        if p.N0 == 0:            # zero forcing: sigma^2 = 0 exactly (the FP64 oracle leaves ~1e-33)
            assert (s2 == 0).all() and np.abs(o["sigma2"]).max() < 1e-20, (idx, s2[:2], o["sigma2"][:2])
            es = 0.0
        else:
            es, _ = parity.check(f"sigma2[{idx}]", s2, o["sigma2"], tol)
        assert ez <= tol and es <= tol, (idx, p.B, p.U, p.C, p.n_sym, ez, es)
        if run.bits:
            L = out["llr"][it.llr_off:it.llr_off + n * NS * U * run.bits].reshape(n, NS, U, run.bits)
            if p.N0 == 0:                 # sigma^2 = 0: infinite LLRs, compare the decisions
                assert (np.sign(L) == np.sign(ollr.maxlog_llr(o["z"], np.ones_like(o["sigma2"])[:, None, :],
                                                               run.bits, p.Es))).all(), (idx, "llr signs")
            else:
                Lo = ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], run.bits, p.Es)
                parity.check(f"llr[{idx}]", L, Lo, 4 * tol)
        if run.cfg.info_elems:
            Ceff = p.C if run.arch == 1 else 1
            info = out["info"][it.info_off:it.info_off + n * Ceff]
            assert (info == 0).all(), (idx, info)
        worst = max(worst, ez)
    return worst


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_uneven_4096_fp32_matches_the_oracle(ff, uneven, arch):
    run = Run(ff, uneven, arch, precision=0)
    run.equalize()
    assert ff.ffeq_device_status() == 0
    _check(run, run.host(), precision=0)


@pytest.mark.parametrize("precision", [1, 2, 3], ids=["TF32X3", "BF16X3", "FP16X3"])
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_uneven_tensor_core_precisions(ff, uneven, arch, precision):
    ps = uneven[:1024]
    run = Run(ff, ps, arch, precision=precision)
    run.equalize()
    assert ff.ffeq_device_status() == 0
    _check(run, run.host(), precision=precision)


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_literal_estimate_and_no_llr(ff, uneven, arch):
    ps = uneven[:300]
    run = Run(ff, ps, arch, estimate=1, llr_bits=0, with_info=False)
    run.equalize()
    _check(run, run.host(), estimate=1)


def test_multi_subcarrier_instances_and_edge_shapes(ff):
    """Several subcarriers per instance, an empty instance, odd B (plain-load
    staging), U = 1, n_sym = 16, S < U, C = 3, Es != 1 and a noiseless one."""
    shapes = [  # B, U, C, n_sc, n_sym, snr, Es
        (64, 16, 4, 37, 14, 10.0, 1.0), (32, 4, 2, 0, 1, 10.0, 1.0), (48, 7, 3, 5, 3, 5.0, 2.0),
        (16, 1, 1, 9, 2, 12.0, 1.0), (128, 32, 16, 3, 16, 20.0, 1.0), (256, 9, 8, 2, 1, 15.0, 0.5),
        (96, 12, 12, 4, 5, 8.0, 1.0), (40, 5, 2, 6, 4, 10.0, 1.0)]
    ps = [synth.make_problem(B, U, C, n, ns, snr_db=snr, bits=4, seed=100 + i, Es=Es)
          for i, (B, U, C, n, ns, snr, Es) in enumerate(shapes)]
    ps.append(synth.make_problem(64, 8, 2, 7, 3, bits=4, seed=7, noiseless=True))
    for arch in (0, 1):
        run = Run(ff, ps, arch)
        run.equalize()
        assert ff.ffeq_device_status() == 0
        _check(run, run.host())
    # Odd B stages with plain loads; odd offsets too.
    odd = [synth.make_problem(B, U, C, 3, ns, bits=4, seed=200 + B) for (B, U, C, ns) in
           [(33, 5, 3, 2), (63, 16, 7, 4), (17, 3, 1, 1)]]
    for arch in (0, 1):
        run = Run(ff, odd, arch)
        run.equalize()
        _check(run, run.host())


def test_every_tuning_gives_identical_bits(ff, uneven):
    ps = uneven[:512]
    for arch in (0, 1):
        run = Run(ff, ps, arch, precision=2)
        run.equalize()
        ref = run.host()
        base = ff.ffeq_batch_get_tuning(run.batch)
        tried = 0
        for gi, (UP, stages, threads, lpr) in enumerate(base):
            for st in (1, 2, 3):
                for th in (64, 128, 256, 512):
                    for lp in (1, 2):
                        t = list(base)
                        t[gi] = (UP, st, th, lp)
                        try:
                            ff.ffeq_batch_set_tuning(run.batch, t)
                        except ff.FfeqError:
                            continue
                        run.z.fill_(complex("nan"))
                        run.equalize()
                        out = run.host()
                        tried += 1
                        if lp == lpr:
                            for k in ("z", "s2", "llr", "info"):
                                np.testing.assert_array_equal(out[k], ref[k], err_msg=f"{k} tuning {t}")
                        else:
                            # Lanes per row change the solve's rounding order only.
                            np.testing.assert_array_equal(out["info"], ref["info"])
                            for k in ("z", "s2"):
                                fin = np.isfinite(ref[k])
                                err = np.abs(out[k][fin] - ref[k][fin]).max() / np.abs(ref[k][fin]).max()
                                assert err <= 1e-5, (k, t, err)
            ff.ffeq_batch_set_tuning(run.batch, base)
        assert tried >= 6


def test_autotune_and_cuda_graph_replay(ff, uneven):
    ps = uneven[:2048]
    run = Run(ff, ps, 1, precision=2)
    ff.ffeq_batch_autotune(run.batch, *run.args(), reps=3)
    run.equalize()
    ref = run.host()
    _check(run, ref, precision=2)
    # Capture on a side stream (the tables are already in the workspace).
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        run.equalize(stream=s)          # warm-up on the capture stream
        s.synchronize()
        run.z.fill_(complex("nan"))      # gaps between instances stay NaN, as in ref
        run.s2.fill_(float("nan"))
        with torch.cuda.graph(g, stream=s):
            run.equalize(stream=s)
    g.replay()
    out = run.host()
    for k in ("z", "s2", "llr", "info"):
        np.testing.assert_array_equal(out[k], ref[k])
    # New inputs of the same sizes and noise levels in the same buffers: the replay follows them.
    ps2 = [synth.make_problem(p.B, p.U, p.C, p.n_sc, p.n_sym, snr_db=p.snr_db, bits=4, seed=50_000 + i)
           for i, p in enumerate(ps)]
    H2, y2 = _flat(ps2, run.cfg, run.inst)
    run.H.copy_(torch.from_numpy(H2))
    run.y.copy_(torch.from_numpy(y2))
    g.replay()
    out = run.host()
    run.ps = ps2
    _check(run, out, precision=2)


def test_corrupted_descriptors_are_skipped_and_reported(ff):
    """Descriptors overwritten in the workspace fail the device checks: the unit
    is skipped, the status word says invalid argument, nothing else changes."""
    ps = [synth.make_problem(64, 8, 2, 4, 2, bits=4, seed=s) for s in range(3)]
    run = Run(ff, ps, 1)
    run.equalize()
    ref = run.host()
    assert ff.ffeq_device_status() == 0
    # Gram-order descriptors start 256 bytes into the workspace, 88 bytes each
    # (seven int64 offsets, then B, U, Ceff, n_sym, N0, rho, llr_scale, inst).
    # First unit: more users than the group's padding; second: channel offset past the end.
    ws = run.ws.cpu().numpy()
    ws[256 + 60:256 + 64].view(np.int32)[0] = 40
    ws[256 + 88:256 + 96].view(np.int64)[0] = run.cfg.h_elems
    run.ws.copy_(torch.from_numpy(ws))
    run.z.fill_(complex("nan"))
    run.equalize()
    out = run.host()
    assert ff.ffeq_device_status() == 1      # FFEQ_ERR_INVALID_ARG
    # Solve-order descriptors are intact, so every z is still produced (from the
    # stale Gram data of the skipped units, which the previous call left in place).
    np.testing.assert_array_equal(out["z"], ref["z"])


def test_tuning_cache_roundtrip(ff, uneven, tmp_path):
    from paper_1808_04473_gb300 import tuning
    ps = uneven[:256]
    path = str(tmp_path / "tuning.json")
    a = Run(ff, ps, 0, precision=2)
    t1, cached1 = tuning.autotune_cached(a.batch, *a.args(), reps=2, path=path)
    assert not cached1
    b = Run(ff, ps, 0, precision=2)
    t2, cached2 = tuning.autotune_cached(b.batch, *b.args(), reps=2, path=path)
    assert cached2 and t2 == t1
    b.equalize()
    _check(b, b.host(), precision=2)


def _linear_instances(eq, seed):
    """Random instances for the ZF / MRC batches: ZF with every inverted Gram
    matrix well posed (B >= 2U for PD, clusters of at least 2U antennas for FD);
    MRC over the whole uneven range plus noiseless instances (one user alone, and
    users on disjoint antennas: the N0 -> 0 limit weights, sigma^2 = 0)."""
    rng = np.random.default_rng(seed)
    ps = []
    for k in range(48):
        B = int(rng.choice([64, 128, 256]))
        if eq == 1:
            U = int(rng.integers(2, 17))
            Cs = [c for c in (1, 2, 4, 8) if B // c >= 2 * U]
        else:
            U = int(rng.integers(1, 33))
            Cs = [c for c in (1, 2, 4, 8, 16) if B // c >= 4]
        C = int(rng.choice(Cs))
        ps.append(synth.make_problem(B, U, C, int(rng.integers(1, 4)), int(rng.integers(1, 15)),
                                     snr_db=float(rng.uniform(5, 20)), bits=4, seed=seed * 1000 + k))
    if eq == 2:
        ps.append(synth.make_problem(64, 1, 4, 3, 5, snr_db=10.0, bits=4, seed=seed + 1, noiseless=True))
        q = synth.make_problem(64, 4, 4, 2, 6, snr_db=10.0, bits=4, seed=seed + 2, noiseless=True)
        for u in range(4):                     # user u only on antennas 16u .. 16u + 15
            mask = np.zeros(64, bool)
            mask[16 * u:16 * u + 16] = True
            q.H[:, u, ~mask] = 0
        q.y[:] = np.einsum("kub,kn u->knb".replace(" ", ""), q.H, np.ones((q.n_sc, q.n_sym, 4), np.complex64))
        ps.append(q)
    return ps


@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("eq", [1, 2], ids=["ZF", "MRC"])
def test_zf_and_mrc_batches_match_the_oracle(ff, arch, eq):
    """ZF and MRC in the uneven batch (``ffeq_batch_config.equalizer``) against
    ``oracle.linear`` per instance: z, sigma^2 and the LLRs (4x) within the BF16x3
    bound, or the kappa-aware bound for ZF (rho = 0)."""
    ps = _linear_instances(eq, seed=7 + arch)
    run = Run(ff, ps, arch, precision=2, llr_bits=4, equalizer=eq)
    run.equalize()
    out = run.host()
    assert ff.ffeq_device_status(clear=True) == 0
    name = "zf" if eq == 1 else "mrc"
    f = olinear.equalize_pd_linear if arch == 0 else olinear.equalize_fd_linear
    for idx, (p, it) in enumerate(zip(ps, run.inst)):
        o = f(p.H, p.y, float(np.float32(p.N0)), p.Es, p.C, name)
        tol = PREC_TOL[2]
        if eq == 1:
            parts = lmmse.partition(p.B, p.C) if arch == 1 else [(0, p.B)]
            kap = max(np.linalg.cond(p.H[k].astype(np.complex128).T[b0:b1].conj().T
                                     @ p.H[k].astype(np.complex128).T[b0:b1])
                      for k in range(p.n_sc) for b0, b1 in parts)
            tol = max(tol, 2.0 * UNIT[2] * kap)
        n, U, NS = p.n_sc, p.U, p.n_sym
        z = out["z"][it.z_off:it.z_off + n * NS * U].reshape(n, NS, U)
        s2 = out["s2"][it.sigma2_off:it.sigma2_off + n * U].reshape(n, U)
        parity.check(f"z[{idx}]", z, o["z"], tol)
        if p.N0 == 0 and eq == 2:
            assert np.array_equal(s2 == 0, o["sigma2"] == 0), idx
        parity.check(f"sigma2[{idx}]", s2, o["sigma2"], tol)
        L = out["llr"][it.llr_off:it.llr_off + n * NS * U * 4].reshape(n, NS, U, 4)
        if p.N0 > 0:
            parity.check(f"llr[{idx}]", L, ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], 4, p.Es), 4 * tol)
        Ceff = p.C if arch == 1 else 1
        assert (out["info"][it.info_off:it.info_off + n * Ceff] == 0).all(), idx


LAMA_TOL = {0: 2e-5, 2: 3e-4, 3: 5e-5}      # the uniform LAMA path's bounds (FP32, BF16x3, FP16x3)


@pytest.mark.parametrize("precision", [0, 2, 3], ids=["fp32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
def test_lama_batch_matches_the_oracle(ff, arch, precision):
    """LAMA (Sec. III-B, Algorithm 1, T = 6) in the uneven batch against
    ``oracle.lama`` per instance: z, sigma^2 per received vector and the LLRs (4x),
    within the uniform LAMA path's bound for the preprocessing precision, on
    instances whose every cluster has beta_c = U / S_c <= 1/2 (as the uniform
    LAMA cases)."""
    rng = np.random.default_rng(11 + arch)
    ps = []
    for k in range(40):
        B = int(rng.choice([64, 128, 256]))
        U = int(rng.integers(1, 33))
        Cs = [c for c in (1, 2, 4, 8, 16) if B // c >= 2 * U]
        if not Cs:
            U = B // 2
            Cs = [1]
        C = int(rng.choice(Cs))
        ps.append(synth.make_problem(B, U, C, int(rng.integers(1, 4)), int(rng.integers(1, 15)),
                                     snr_db=float(rng.uniform(5, 20)), bits=4, seed=9000 + 100 * arch + k,
                                     Es=float(rng.choice([1.0, 2.0]))))
    run = Run(ff, ps, arch, precision=precision, llr_bits=4, equalizer=ff.LAMA, lama_iters=6)
    run.equalize()
    out = run.host()
    assert ff.ffeq_device_status(clear=True) == 0
    f = olama.equalize_pd_lama if arch == 0 else olama.equalize_fd_lama
    tol = LAMA_TOL[precision]
    for idx, (p, it) in enumerate(zip(ps, run.inst)):
        o = f(p.H, p.y, float(np.float32(p.N0)), p.Es, p.C, 4, 6)
        n, U, NS = p.n_sc, p.U, p.n_sym
        z = out["z"][it.z_off:it.z_off + n * NS * U].reshape(n, NS, U)
        s2 = out["s2"][it.sigma2_off:it.sigma2_off + n * NS * U].reshape(n, NS, U)
        parity.check(f"z[{idx}]", z, o["z"], tol)
        parity.check(f"sigma2[{idx}]", s2, o["sigma2"], tol)
        L = out["llr"][it.llr_off:it.llr_off + n * NS * U * 4].reshape(n, NS, U, 4)
        parity.check(f"llr[{idx}]", L, ollr.maxlog_llr(o["z"], o["sigma2"], 4, p.Es), 4 * tol)
        Ceff = p.C if arch == 1 else 1
        assert (out["info"][it.info_off:it.info_off + n * Ceff] == 0).all(), idx
