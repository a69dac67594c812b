"""C-ABI checks that need no GPU: the library builds, loads, exports every symbol
declared in include/ffeq.h, and rejects bad arguments before touching CUDA."""
import ctypes
import re
import os
import subprocess

import pytest

from paper_1808_04473_gb300 import build as fbuild
from paper_1808_04473_gb300 import ffeq


@pytest.fixture(scope="module")
def built():
    fbuild.build()
    return ffeq.lib()


def test_library_exports_every_header_symbol(built):
    names = ffeq.header_symbols()
    assert "ffeq_equalize" in names and "ffeq_plan_create" in names
    for n in names:
        assert hasattr(built, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", ffeq.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_version_and_status_strings(built):
    assert ffeq.ffeq_version() >= 100
    assert ffeq.ffeq_status_string(0) == "ok"
    assert "invalid" in ffeq.ffeq_status_string(1)


@pytest.mark.parametrize("kw,status", [
    (dict(B=0, U=4, C=1), 1), (dict(B=32, U=4, C=3), 1), (dict(B=32, U=0, C=2), 1),
    (dict(B=32, U=4, C=2, arch=7), 1), (dict(B=32, U=4, C=2, estimate=5), 1),
    (dict(B=32, U=4, C=2, llr_bits=3), 1), (dict(B=32, U=4, C=2, precision=9), 1),
    (dict(B=32, U=4, C=2, precision=4), 1),
    (dict(B=32, U=33, C=2), 2), (dict(B=32, U=4, C=2, n_sym=17), 2), (dict(B=8192, U=32, C=2), 2),
])
def test_plan_validation(built, kw, status):
    args = dict(B=32, U=4, C=2, n_sc=8, n_sym=1)
    args.update(kw)
    with pytest.raises(ffeq.FfeqError) as e:
        ffeq.ffeq_plan_create(**args)
    assert e.value.status == status


def test_equalize_rejects_bad_arguments_without_cuda(built):
    plan = ffeq.ffeq_plan_create(32, 4, 2, 8, 1)
    fake = 1 << 20                                  # never dereferenced: validation fails first
    for N0, Es in ((-1.0, 1.0), (1.0, 0.0), (float("nan"), 1.0), (1.0, float("inf"))):
        with pytest.raises(ffeq.FfeqError) as e:
            ffeq.ffeq_equalize(plan, fake, fake, N0, Es, fake, fake, workspace=fake, workspace_bytes=1 << 30,
                               stream=0)
        assert e.value.status == 1
    with pytest.raises(ffeq.FfeqError):
        ffeq.ffeq_equalize(plan, None, fake, 1.0, 1.0, fake, fake, workspace=fake, workspace_bytes=1 << 30,
                           stream=0)
    with pytest.raises(ffeq.FfeqError):                                         # misaligned H
        ffeq.ffeq_equalize(plan, fake + 4, fake, 1.0, 1.0, fake, fake, workspace=fake, workspace_bytes=1 << 30,
                           stream=0)
    need = ffeq.ffeq_workspace_size(plan)
    with pytest.raises(ffeq.FfeqError):                                         # workspace too small
        ffeq.ffeq_equalize(plan, fake, fake, 1.0, 1.0, fake, fake, workspace=fake, workspace_bytes=need - 1,
                           stream=0)
    llr_plan = ffeq.ffeq_plan_create(32, 4, 2, 8, 1, llr_bits=4)
    with pytest.raises(ffeq.FfeqError):
        ffeq.ffeq_equalize(llr_plan, fake, fake, 1.0, 1.0, fake, fake, llr=None, workspace=fake,
                           workspace_bytes=1 << 30, stream=0)
    empty = ffeq.ffeq_plan_create(32, 4, 2, 0, 1)                                # n_sc = 0 is a no-op
    ffeq.ffeq_equalize(empty, None, None, 1.0, 1.0, None, None, stream=0)


def test_staging_size_accounts_for_every_buffer(built):
    plan = ffeq.ffeq_plan_create(256, 16, 8, 1200, 14, arch=ffeq.FD, llr_bits=4)
    n = ffeq.ffeq_host_staging_size(plan)
    ws = 1200 * 8 * (16 + 14) * 16 * 8
    assert ffeq.ffeq_workspace_size(plan) == ws
    need = 1200 * 16 * 256 * 8 + 1200 * 14 * 256 * 8 + 1200 * 14 * 16 * 8 + 1200 * 16 * 4 + \
        1200 * 14 * 16 * 4 * 4 + 1200 * 8 * 4 + ws
    assert need <= n <= need + 8 * 256
    pd = ffeq.ffeq_plan_create(256, 16, 8, 1200, 14, arch=ffeq.PD)
    assert ffeq.ffeq_workspace_size(pd) == 1200 * (16 + 14) * 16 * 8


def test_plan_struct_layout_matches_header(built):
    assert ctypes.sizeof(ffeq.ffeq_problem) == 13 * 4
    text = open(ffeq.HEADER_PATH).read()
    body = text[text.index("typedef struct {") + len("typedef struct {"):text.index("} ffeq_problem;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = [f.strip() for decl in body.split(";") for f in decl.replace("int", "").split(",") if f.strip()]
    assert fields == [n for n, _ in ffeq.ffeq_problem._fields_]


def test_oracle_and_cuda_sources_are_independent(repo_root):
    """The oracle never imports the CUDA path, and the package never imports the oracle."""
    for dirpath, _, files in os.walk(os.path.join(repo_root, "oracle")):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert "paper_1808_04473_gb300" not in src and "ffeq" not in src.replace("ffeq_", ""), f
    pkg = os.path.join(repo_root, "paper_1808_04473_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_plan_tuning_validation(built):
    ff = ffeq
    plan = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=ff.FP32)
    assert ff.ffeq_plan_get_tuning(plan) == (0, 0)
    # out of range; pre-split, the 4-warp and the streamed shapes need a tensor-core precision
    for bad, status in (((8, 0), 1), ((-1, 0), 1), ((1, 4), 1), ((3, 0), 2), ((4, 0), 2), ((5, 0), 2), ((6, 0), 2),
                        ((7, 0), 2)):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_set_tuning(plan, bad)
        assert e.value.status == status, bad
    assert ff.ffeq_plan_get_tuning(plan) == (0, 0)
    ff.ffeq_plan_set_tuning(plan, (2, 1))
    assert ff.ffeq_plan_get_tuning(plan) == (2, 1)
    # Too deep a pipeline for this problem: three 99 KB stages do not fit.
    big = ff.ffeq_plan_create(256, 32, 16, 10, 16, arch=ff.FD, precision=ff.BF16X3)
    with pytest.raises(ff.FfeqError) as e:
        ff.ffeq_plan_set_tuning(big, (1, 3))
    assert e.value.status == 2
    ff.ffeq_plan_set_tuning(big, (3, 0))
    # The streamed shape: BF16x3 or FP16x3 with whole 16-antenna clusters (FD);
    # its second value is the depth of each subcarrier's ring (0: 3).
    # The half-size streamed shape (7) takes the same problems with the same depths.
    for prec in (ff.BF16X3, ff.FP16X3):
        fd = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=prec)
        for v in (5, 7):
            for st in (0, 2, 3):
                ff.ffeq_plan_set_tuning(fd, (v, st))
                assert ff.ffeq_plan_get_tuning(fd) == (v, st)
            for st, status in ((4, 1), (1, 2)):        # depth 1 cannot convert one slice ahead
                with pytest.raises(ff.FfeqError) as e:
                    ff.ffeq_plan_set_tuning(fd, (v, st))
                assert e.value.status == status
    # The fused shape: the streamed shape's conditions, U = 8 or 16, L-MMSE or ZF
    # without refinement; ring depth 2 (0 means 2).
    for prec in (ff.BF16X3, ff.FP16X3):
        fd = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=prec)
        for st in (0, 2):
            ff.ffeq_plan_set_tuning(fd, (6, st))
            assert ff.ffeq_plan_get_tuning(fd) == (6, st)
        for st in (1, 3):
            with pytest.raises(ff.FfeqError) as e:
                ff.ffeq_plan_set_tuning(fd, (6, st))
            assert e.value.status == 2
    for kw in (dict(U=12), dict(U=32), dict(equalizer=ff.MRC), dict(equalizer=ff.LAMA, lama_iters=2, llr_bits=4),
               dict(refine=1)):
        a = dict(B=256, U=16, C=8, n_sc=10, n_sym=14, arch=ff.FD, precision=ff.BF16X3)
        a.update(kw)
        pl = ff.ffeq_plan_create(a.pop("B"), a.pop("U"), a.pop("C"), a.pop("n_sc"), a.pop("n_sym"), **a)
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_set_tuning(pl, (6, 2))
        assert e.value.status == 2, kw
    odd = ff.ffeq_plan_create(96, 8, 8, 10, 2, arch=ff.FD, precision=ff.BF16X3)      # S = 12
    for v in (5, 6, 7):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_set_tuning(odd, (v, 0))
        assert e.value.status == 2
    ff.ffeq_plan_set_tuning(ff.ffeq_plan_create(96, 8, 8, 10, 2, arch=ff.PD, precision=ff.BF16X3), (5, 0))
    tf = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=ff.TF32X3)
    with pytest.raises(ff.FfeqError) as e:
        ff.ffeq_plan_set_tuning(tf, (5, 0))
    assert e.value.status == 2
    # FP16x3 runs on the 16-warp, streamed, fused and half-size streamed shapes only.
    h = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=ff.FP16X3)
    for v in (2, 3, 4):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_set_tuning(h, (v, 0))
        assert e.value.status == 2, v


def test_autotune_sets_checks_arguments(built):
    plan = ffeq.ffeq_plan_create(64, 8, 4, 10, 2, arch=ffeq.FD, precision=ffeq.BF16X3)
    L = ffeq.lib()
    arr = (ctypes.c_void_p * 1)(256)
    for H, y, n, reps in ((None, arr, 1, 2), (arr, None, 1, 2), (arr, arr, 0, 2), (arr, arr, 1, 0)):
        st = L.ffeq_plan_autotune_sets(plan.handle, H, y, n, 1.0, 1.0, 256, 256, None, None, 256, 1 << 20, None, reps)
        assert st == 1
    with pytest.raises(ValueError):
        ffeq.ffeq_plan_autotune_sets(plan, [], [], 1.0, 1.0, None, None)


def test_refinement_needs_the_inputs(built):
    plan = ffeq.ffeq_plan_create(64, 8, 4, 10, 2, arch=ffeq.FD, precision=ffeq.BF16X3, refine=1)
    plain = ffeq.ffeq_plan_create(64, 8, 4, 10, 2, arch=ffeq.FD, precision=ffeq.BF16X3)
    assert ffeq.ffeq_workspace_size(plan) >= ffeq.ffeq_workspace_size(plain) + 10 * 4 * ((2 + 8) * 8 * 8 + 4)
    with pytest.raises(ffeq.FfeqError) as e:
        ffeq.ffeq_fuse_equalize(plan, 256, ffeq.ffeq_workspace_size(plan), 0.1, 1.0, 256, 256, None, None, stream=0)
    assert e.value.status == 2
    with pytest.raises(ffeq.FfeqError) as e:
        ffeq.ffeq_plan_create(64, 8, 4, 10, 2, refine=5)
    assert e.value.status == 1
    # The FP64 residual is a mode of the refinement: 0..2, and only with refine > 0.
    for bad in (dict(refine=1, refine_fp64=3), dict(refine=1, refine_fp64=-1), dict(refine=0, refine_fp64=1)):
        with pytest.raises(ffeq.FfeqError) as e:
            ffeq.ffeq_plan_create(64, 8, 4, 10, 2, **bad)
        assert e.value.status == 1, bad
    ffeq.ffeq_plan_create(64, 8, 4, 10, 2, arch=ffeq.FD, refine=2, refine_fp64=1)


def test_cluster_sizes_validation(built):
    ff = ffeq
    # C sizes >= 0 summing to B; B % C need not be 0 then.
    ff.ffeq_plan_create(100, 8, 3, 10, 2, arch=ff.FD, cluster_sizes=[40, 35, 25])
    ff.ffeq_plan_create(128, 8, 3, 10, 2, arch=ff.FD, cluster_sizes=[64, 0, 64])
    ff.ffeq_plan_create(100, 8, 3, 10, 2, arch=ff.PD, cluster_sizes=[40, 35, 25])
    for sizes in ([40, 35, 24], [40, 35, 26], [50, -5, 55]):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_create(100, 8, 3, 10, 2, arch=ff.FD, cluster_sizes=sizes)
        assert e.value.status == 1, sizes
    with pytest.raises(ff.FfeqError) as e:                     # B % C != 0 needs sizes
        ff.ffeq_plan_create(100, 8, 3, 10, 2, arch=ff.FD)
    assert e.value.status == 1
    with pytest.raises(ValueError):
        ff.ffeq_plan_create(100, 8, 3, 10, 2, arch=ff.FD, cluster_sizes=[50, 50])
    # Unequal FD clusters: the streamed and pre-split shapes do not apply.
    fd = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=ff.BF16X3,
                             cluster_sizes=[16, 48, 32, 32, 32, 32, 32, 32])
    for v in (3, 5):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_set_tuning(fd, (v, 0))
        assert e.value.status == 2, v
    ff.ffeq_plan_set_tuning(fd, (1, 0))
    # Equal sizes given explicitly are the uniform plan (the streamed shape applies).
    eq = ff.ffeq_plan_create(256, 16, 8, 10, 14, arch=ff.FD, precision=ff.BF16X3, cluster_sizes=[32] * 8)
    ff.ffeq_plan_set_tuning(eq, (5, 0))
    # The training entry points take the plan's clusters; their argument checks
    # come before any device call (a workspace below ffeq_fd_train_workspace_size).
    L = ff.lib()
    st = L.ffeq_fd_train_forward(fd.handle, 256, 256, 256, 256, 256, 256, 16, None)
    assert st == 1


def test_equalizer_validation(built):
    ff = ffeq
    for eq in (ff.LMMSE, ff.ZF, ff.MRC):
        for arch in (ff.PD, ff.FD):
            ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=arch, precision=ff.BF16X3, equalizer=eq)
    for bad in (-1, 3):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_create(64, 8, 4, 10, 2, equalizer=bad)
        assert e.value.status == 1
    # Refinement of a solve: L-MMSE and ZF; MRC solves nothing.
    ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=ff.FD, refine=1, equalizer=ff.ZF)
    with pytest.raises(ff.FfeqError) as e:
        ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=ff.FD, refine=1, equalizer=ff.MRC)
    assert e.value.status == 1
    # The differentiable FD form is L-MMSE (checked before any device call).
    for eq in (ff.ZF, ff.MRC):
        fd = ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=ff.FD, equalizer=eq)
        assert ff.lib().ffeq_fd_train_forward(fd.handle, 256, 256, 256, 256, 256, 256, 1 << 30, None) == 2


def test_lama_validation(built):
    ff = ffeq
    for arch in (ff.PD, ff.FD):
        ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=arch, llr_bits=4, equalizer=ff.LAMA, lama_iters=8)
    bad = [dict(llr_bits=0, lama_iters=8),                 # the prior is the LLR constellation
           dict(llr_bits=4, lama_iters=0), dict(llr_bits=4, lama_iters=65),
           dict(llr_bits=4, lama_iters=8, refine=1)]
    for kw in bad:
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=ff.FD, equalizer=ff.LAMA, **kw)
        assert e.value.status == 1, kw
    with pytest.raises(ff.FfeqError) as e:                    # iterations only for LAMA
        ff.ffeq_plan_create(64, 8, 4, 10, 2, lama_iters=3)
    assert e.value.status == 1
    # N0 = 0 is rejected before any device work (the denoiser needs tau > 0).
    plan = ff.ffeq_plan_create(32, 4, 2, 8, 1, llr_bits=2, equalizer=ff.LAMA, lama_iters=4)
    fake = 1 << 20
    with pytest.raises(ff.FfeqError) as e:
        ff.ffeq_fuse_equalize(plan, fake, 1 << 30, 0.0, 1.0, fake, fake, fake, None, stream=0)
    assert e.value.status == 1
    # sigma2 holds one value per received vector: the host staging counts n_sc * n_sym * U floats.
    lm = ff.ffeq_plan_create(256, 16, 8, 100, 14, arch=ff.FD, llr_bits=4, equalizer=ff.LAMA, lama_iters=8)
    mm = ff.ffeq_plan_create(256, 16, 8, 100, 14, arch=ff.FD, llr_bits=4, equalizer=ff.MRC)
    assert ff.ffeq_host_staging_size(lm) - ff.ffeq_host_staging_size(mm) >= 100 * 13 * 16 * 4


def test_plain_c_client_compiles_links_and_runs(built, tmp_path):
    """The headers are plain C (C11, -Wall -Werror) and a C program linked against
    libffeq.so makes host-side calls through them without a GPU."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "abi_check")
    libdir = os.path.dirname(ffeq.LIB_PATH)
    cc = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", ffeq.INCLUDE_DIR,
                         os.path.join(root, "tests", "c", "abi_check.c"), "-o", exe, "-L", libdir, "-lffeq",
                         "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stderr


def test_optimal_backward_validation(built):
    """ffeq_fd_optimal_backward differentiates the FD estimate with unbiased pairs and
    no refinement: other plans are rejected before any launch; the workspace holds the
    contraction output, G_b and the H-term matrices."""
    ff = ffeq
    ok = ff.ffeq_plan_create(64, 8, 4, 10, 2, arch=ff.FD)
    nb = ff.ffeq_fd_optimal_workspace_size(ok)
    plain = ff.ffeq_workspace_size(ok)
    assert nb >= plain + 10 * 4 * (2 * 8 + 8 * 8) * 8
    for bad in (dict(arch=ff.PD), dict(arch=ff.FD, estimate=ff.LITERAL), dict(arch=ff.FD, refine=1),
                dict(arch=ff.FD, equalizer=ff.ZF)):
        plan = ff.ffeq_plan_create(64, 8, 4, 10, 2, **bad)
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_fd_optimal_workspace_size(plan)
        assert e.value.status == 1, bad
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_fd_optimal_backward(plan, 256, 256, 0.1, 1.0, 256, 256, 256, 256, nb, stream=0)
        assert e.value.status == 1, bad
    # Null buffers, a short workspace and bad scalars are argument errors.
    for args in ((None, 256, 0.1, 1.0, 256, 256, 256, 256, nb), (256, 256, 0.1, 1.0, 256, 256, 256, 256, nb - 1),
                 (256, 256, -1.0, 1.0, 256, 256, 256, 256, nb), (256, 256, 0.1, 0.0, 256, 256, 256, 256, nb)):
        with pytest.raises(ff.FfeqError) as e:
            ff.ffeq_fd_optimal_backward(ok, *args, stream=0)
        assert e.value.status == 1, args
    # Clusters of given sizes are accepted.
    sized = ff.ffeq_plan_create(100, 8, 3, 10, 2, arch=ff.FD, cluster_sizes=[40, 35, 25])
    assert ff.ffeq_fd_optimal_workspace_size(sized) > 0
