"""GPU parity of every launch shape of the uniform plan (include/ffeq.h tuning),
the fused shape 6 and the half-size streamed shape 7 included.

Each contraction shape and pipeline depth that fits is run on the same inputs
and checked against the FP64 oracle with the bounds of test_gpu_parity (1e-5
FP32, 2e-4 BF16x3, 2e-5 FP16x3 per subcarrier and per entry).  (Shapes may split a cluster's antennas
among a different number of warps, so results agree to rounding, not bit for
bit.)  The autotuner returns a shape that fits.
"""
import numpy as np
import pytest

import parity
from oracle import lmmse
from paper_1808_04473_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 2: 2e-4, 3: 2e-5}


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04473_gb300 import build as fbuild
    from paper_1808_04473_gb300 import ffeq
    fbuild.build()
    ffeq.lib()
    return ffeq


@pytest.mark.parametrize("precision", [0, 2, 3], ids=["fp32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("arch", [0, 1], ids=["PD", "FD"])
@pytest.mark.parametrize("shape", [(256, 16, 8, 300, 14), (128, 32, 16, 40, 16), (64, 8, 4, 77, 3),
                                   (96, 12, 2, 50, 5), (48, 3, 3, 20, 1),
                                   # B not a multiple of 16 (PD: the last 16-antenna block of the
                                   # streamed shape is partly the copies' zero fill; FD clusters of 25
                                   # and 10 antennas do not take the streamed shape)
                                   (100, 8, 4, 30, 2), (10, 4, 1, 9, 1)])
def test_every_shape_matches_the_oracle(ff, arch, precision, shape):
    B, U, C, n_sc, n_sym = shape
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=12.0, bits=4, seed=B + U)
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    plan = ff.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=arch, precision=precision)
    nb = ff.ffeq_workspace_size(plan)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    z = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=dev)
    s2 = torch.empty((n_sc, U), dtype=torch.float32, device=dev)
    f = lmmse.equalize_pd if arch == 0 else lmmse.equalize_fd
    o = f(p.H, p.y, float(np.float32(p.N0)), p.Es, C, "unbiased")
    results = {}
    for variant in (1, 2, 3, 4, 5, 6, 7):
        for stages in (0, 1, 2, 3):
            try:
                ff.ffeq_plan_set_tuning(plan, (variant, stages))
            except ff.FfeqError as e:
                assert e.status == 2
                continue
            z.fill_(complex("nan"))
            ff.ffeq_equalize(plan, H, y, p.N0, p.Es, z, s2, None, None, ws, nb)
            torch.cuda.synchronize()
            zn = z.cpu().numpy()
            parity.check(f"z {variant, stages}", zn, o["z"], TOL[precision])
            parity.check(f"sigma2 {variant, stages}", s2.cpu().numpy(), o["sigma2"], TOL[precision])
            results[(variant, stages)] = zn
    assert any(k[0] == 1 for k in results)          # the default shape always fits
    t = ff.ffeq_plan_autotune_sets(plan, [H, H.clone()], [y, y.clone()], p.N0, p.Es, z, s2, None, None, ws, nb,
                                   reps=2)
    assert t[0] in (1, 2, 3, 4, 5, 6, 7) and 1 <= t[1] <= 3
    t = ff.ffeq_plan_autotune(plan, H, y, p.N0, p.Es, z, s2, None, None, ws, nb, reps=2)
    assert t[0] in (1, 2, 3, 4, 5, 6, 7) and 1 <= t[1] <= 3
    if precision != 0 and (arch == 0 or C == 1 or (B // C) % 16 == 0):   # one cluster: no boundaries
        assert (5, 2) in results and (5, 3) in results   # the streamed shape takes every such problem
        assert (7, 2) in results and (7, 3) in results   # and its half-size CTA form (the same sums per warp)
        assert np.array_equal(results[(7, 3)].view(np.int32), results[(5, 3)].view(np.int32))
        # the fused one where the users fill a lane group (the same bits as shape 5, ring 2)
        assert ((6, 2) in results) == (U in (8, 16))
        if (6, 2) in results:
            assert np.array_equal(results[(6, 2)].view(np.int32), results[(5, 2)].view(np.int32))
    else:
        assert not any(k[0] in (5, 6, 7) for k in results)
    assert ff.ffeq_plan_get_tuning(plan) == t
