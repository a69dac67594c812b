"""The allocation-free entry point against the regular one (GPU).

ffeq_equalize_noalloc exists for callers that cannot allocate device memory
(a real-time receive chain that must not enter the CUDA allocator, a plug-in
that owns no device memory): it takes its workspace from an array compiled
into the library.  Two calls in a row must each match ffeq_equalize, which is
given a workspace of its own: bit for bit, since both run the same kernels.
This file is collected last so that a stop at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

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


def _run(ff, p, arch, noalloc):
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    plan = ff.ffeq_plan_create(p.B, p.U, p.C, p.n_sc, p.n_sym, arch=arch, llr_bits=p.bits)
    z = torch.empty((p.n_sc, p.n_sym, p.U), dtype=torch.complex64, device=dev)
    s2 = torch.empty((p.n_sc, p.U), dtype=torch.float32, device=dev)
    L = torch.empty((p.n_sc, p.n_sym, p.U, p.bits), dtype=torch.float32, device=dev)
    info = torch.empty((p.n_sc, p.C if arch == ff.FD else 1), dtype=torch.int32, device=dev)
    if noalloc:
        ff.ffeq_equalize_noalloc(plan, H, y, p.N0, p.Es, z, s2, L, info)
    else:
        nb = ff.ffeq_workspace_size(plan)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        ff.ffeq_equalize(plan, H, y, p.N0, p.Es, z, s2, L, info, ws, nb)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in dict(z=z, s2=s2, L=L, info=info).items()}


def test_noalloc_matches_workspace_path_on_two_calls_in_a_row(ff):
    # Two different problems back to back through the shared array: the second
    # call must not see anything left over from the first.  Both entry points
    # run the same kernels in the same order on the same inputs, so the outputs
    # are equal bit for bit (which is within any tolerance of the GPU tests).
    cases = [(synth.make_problem(256, 16, 8, 600, 14, snr_db=12.0, bits=4, seed=31), ff.FD),
             (synth.make_problem(128, 12, 4, 300, 7, snr_db=6.0, bits=2, seed=32), ff.PD)]
    for p, arch in cases:
        got = _run(ff, p, arch, noalloc=True)
        ref = _run(ff, p, arch, noalloc=False)
        for key in ("z", "s2", "L", "info"):
            assert np.array_equal(got[key], ref[key]), key
    assert ff.ffeq_device_status() == 0


def test_noalloc_rejects_problems_beyond_the_fixed_array(ff):
    # FD workspace of 6000 x 8 x (16 + 14) x 16 x 8 bytes = 184 MB > 64 MiB.
    plan = ff.ffeq_plan_create(256, 16, 8, 6000, 14, arch=ff.FD)
    with pytest.raises(ff.FfeqError) as e:
        ff.ffeq_equalize_noalloc(plan, 1 << 20, 1 << 20, 1.0, 1.0, 1 << 20, 1 << 20)
    assert e.value.status == 2
