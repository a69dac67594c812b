"""The fused shape (tuning value 6 in include/ffeq.h): the streamed contraction
with the solve, the optimal fusion and the soft outputs in the same launch.

Per lane the fused kernel does the arithmetic of the separate launches (the
streamed contraction with a ring of 2, then the solve kernel: the same sweep,
the same right-hand-side products and the fusion terms summed in cluster
order), so ffeq_equalize must give the SAME BITS under tuning (6, 2) and (5, 2):
z, sigma^2, the LLRs and the info codes, including NaN outputs of a failed
factorization.  The cases cover PD and FD, U = 8 and 16, both 16-bit split
precisions, L-MMSE (unbiased and literal) and ZF, 1 to 16 symbols, problems with
fewer subcarriers than lane groups (idle groups) and with more than one
subcarrier per group (the handoff buffers' phases over several subcarriers), and
PD with B not a multiple of 16.  The fused outputs are also checked against the
FP64 oracle with the bounds of test_gpu_parity, and the split entry points
under shape 6 (ffeq_local_preprocess + ffeq_fuse_equalize) against the fused
call.
"""
import numpy as np
import pytest

import parity
from oracle import linear as olinear
from oracle import llr as ollr
from oracle import lmmse
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {2: 2e-4, 3: 2e-5}


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


def _run(ff, plan, H, y, N0, Es, shape, bits, tuning, split=False):
    B, U, C, n_sc, n_sym = shape
    dev = H.device
    ff.ffeq_plan_set_tuning(plan, tuning)
    nb = ff.ffeq_workspace_size(plan)
    ws = torch.empty(max(nb, 16), dtype=torch.uint8, device=dev)
    z = torch.full((n_sc, n_sym, U), complex("nan"), dtype=torch.complex64, device=dev)
    s2 = torch.full((n_sc, U), -1.0, dtype=torch.float32, device=dev)
    llr = torch.full((n_sc, n_sym, U, bits), -7.0, dtype=torch.float32, device=dev) if bits else None
    Ceff = C if plan.problem.arch == ff.FD else 1
    info = torch.full((n_sc, Ceff), -5, dtype=torch.int32, device=dev)
    if split:
        ff.ffeq_local_preprocess(plan, H, y, ws, nb)
        ff.ffeq_fuse_equalize(plan, ws, nb, N0, Es, z, s2, llr, info)
    else:
        ff.ffeq_equalize(plan, H, y, N0, Es, z, s2, llr, info, ws, nb)
    torch.cuda.synchronize()
    assert ff.ffeq_device_status(clear=True) == 0
    out = {"z": z, "sigma2": s2, "info": info}
    if bits:
        out["llr"] = llr
    return out


def _same_bits(a, b):
    for k in a:
        x, y = a[k].contiguous(), b[k].contiguous()
        xi = x.view(torch.int32) if x.dtype != torch.complex64 else torch.view_as_real(x).view(torch.int32)
        yi = y.view(torch.int32) if y.dtype != torch.complex64 else torch.view_as_real(y).view(torch.int32)
        assert torch.equal(xi, yi), k


CASES = [
    # (B, U, C, n_sc, n_sym), arch, precision, equalizer, estimate, bits
    ((256, 16, 8, 300, 14), 1, 2, 0, 0, 4),
    ((256, 16, 8, 300, 14), 0, 2, 0, 0, 4),
    ((256, 16, 8, 2500, 14), 1, 3, 0, 0, 6),      # more subcarriers than lane groups
    ((256, 16, 8, 2500, 14), 0, 3, 0, 0, 2),
    ((128, 8, 4, 77, 3), 1, 2, 0, 1, 4),
    ((128, 8, 4, 77, 3), 0, 3, 0, 1, 0),
    ((64, 16, 1, 50, 16), 1, 2, 0, 0, 4),         # FD with one cluster
    ((100, 16, 4, 30, 2), 0, 2, 0, 0, 4),         # PD, B not a multiple of 16
    ((256, 16, 8, 5, 1), 1, 3, 0, 0, 4),          # fewer subcarriers than CTAs x teams
    ((256, 16, 8, 300, 7), 1, 2, 1, 0, 4),        # ZF
    ((512, 8, 16, 1300, 14), 1, 3, 0, 0, 4),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{'PD' if c[1] == 0 else 'FD'}-p{c[2]}-eq{c[3]}-est{c[4]}-b{c[5]}"
                                             for c in CASES])
def test_fused_matches_separate_launches_and_oracle(ff, case):
    shape, arch, prec, eq, est, bits = case
    B, U, C, n_sc, n_sym = shape
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=12.0, bits=bits or 4, seed=B + U + n_sc)
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    plan = ff.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=arch, precision=prec, estimate=est, llr_bits=bits,
                               equalizer=eq)
    fused = _run(ff, plan, H, y, p.N0, p.Es, shape, bits, (6, 2))
    separate = _run(ff, plan, H, y, p.N0, p.Es, shape, bits, (5, 2))
    _same_bits(fused, separate)
    split = _run(ff, plan, H, y, p.N0, p.Es, shape, bits, (6, 0), split=True)
    _same_bits(fused, split)
    # FP64 oracle on a sample of subcarriers.
    idx = np.unique(np.linspace(0, n_sc - 1, min(n_sc, 40)).astype(int))
    N0 = float(np.float32(p.N0))
    if eq == 1:
        f = olinear.equalize_pd_linear if arch == 0 else olinear.equalize_fd_linear
        o = f(p.H[idx], p.y[idx], N0, p.Es, C, "zf")
    else:
        f = lmmse.equalize_pd if arch == 0 else lmmse.equalize_fd
        o = f(p.H[idx], p.y[idx], N0, p.Es, C, "unbiased" if est == 0 else "literal")
    z = fused["z"].cpu().numpy()[idx]
    s2 = fused["sigma2"].cpu().numpy()[idx]
    tol = TOL[prec] * (10 if eq == 1 else 1)      # ZF: no regularization, larger condition numbers
    parity.check("z", z, o["z"], tol)
    parity.check("sigma2", s2, o["sigma2"], tol)
    assert (fused["info"].cpu().numpy() == 0).all()
    if bits:
        lo = ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], bits, p.Es)
        parity.check("llr", fused["llr"].cpu().numpy()[idx], lo, 4 * tol)


def test_fused_failed_factorization_gives_the_same_nans(ff):
    """ZF where a cluster cannot see a user: G_c has a zero row and column, the
    sweep meets the pivot 0 at that user, and both launches report the same info
    codes and NaN outputs (the clusters with S < U do not take the streamed
    shapes at all)."""
    B, U, C, n_sc, n_sym = 64, 16, 8, 40, 4          # S = 8 < U = 16
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=12.0, bits=4, seed=3)
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    plan = ff.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ff.FD, precision=ff.BF16X3, llr_bits=4, equalizer=ff.ZF)
    with pytest.raises(ff.FfeqError):     # S = 8: not whole 16-antenna clusters, the streamed shapes do not apply
        ff.ffeq_plan_set_tuning(plan, (6, 2))
    B = 256                                           # S = 32 antennas per cluster
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=12.0, bits=4, seed=4)
    Hn = p.H.copy()
    Hn[::3, 5, :32] = 0          # user 5 unseen by cluster 0 of every third subcarrier: G_0 has a zero row and column
    H = torch.from_numpy(Hn).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    plan = ff.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ff.FD, precision=ff.BF16X3, llr_bits=4, equalizer=ff.ZF)
    shape = (B, U, C, n_sc, n_sym)
    fused = _run(ff, plan, H, y, p.N0, p.Es, shape, 4, (6, 2))
    separate = _run(ff, plan, H, y, p.N0, p.Es, shape, 4, (5, 2))
    _same_bits(fused, separate)
    info = fused["info"].cpu().numpy()
    assert (info[::3, 0] == 6).all() and (info[1::3] == 0).all()
    assert np.isnan(fused["z"].cpu().numpy()[::3]).all()


def test_fused_shape_applies_to_lmmse_and_zf_without_refinement(ff):
    for kw, ok in ((dict(), True), (dict(equalizer=1), True), (dict(equalizer=2), False),
                   (dict(refine=1), False), (dict(precision=0), False)):
        args = dict(arch=ff.FD, precision=ff.BF16X3)
        args.update(kw)
        plan = ff.ffeq_plan_create(256, 16, 8, 10, 14, **args)
        if ok:
            ff.ffeq_plan_set_tuning(plan, (6, 2))
            assert ff.ffeq_plan_get_tuning(plan) == (6, 2)
        else:
            with pytest.raises(ff.FfeqError) as e:
                ff.ffeq_plan_set_tuning(plan, (6, 2))
            assert e.value.status == 2, kw
