"""Host-side logic of uneven batches (include/ffeq_batch.h), without a GPU.

Plan creation validates every instance and builds the schedule on the host;
these tests check the argument checks, the grouping by padded users, the
workspace size and the tuning interface.  No call here launches a kernel.
"""
import pytest

from paper_1808_04473_gb300 import synth

ffeq = pytest.importorskip("paper_1808_04473_gb300.ffeq")


@pytest.fixture(scope="module")
def lib():
    from paper_1808_04473_gb300 import build as fbuild
    fbuild.build()
    return ffeq.lib()


def _specs(ps):
    return [(p.B, p.U, p.C, p.n_sc, p.n_sym, p.N0, p.Es) for p in ps]


def _status(fn, *a, **k):
    try:
        fn(*a, **k)
    except ffeq.FfeqError as e:
        return e.status
    return 0


def test_groups_by_padded_users_and_workspace_size(lib):
    ps = synth.make_uneven(512, seed=2)
    for arch in (ffeq.PD, ffeq.FD):
        cfg, inst = ffeq.pack_batch(_specs(ps), arch=arch, llr_bits=4)
        b = ffeq.ffeq_batch_create(cfg, inst)
        tun = ffeq.ffeq_batch_get_tuning(b)
        ups = {8 if p.U <= 8 else 16 if p.U <= 16 else 32 for p in ps}
        assert {t[0] for t in tun} == ups
        for UP, stages, threads, lpr in tun:
            assert 1 <= stages <= 3 and threads % 32 == 0 and 32 <= threads <= 512 and lpr in (1, 2)
            assert lpr == (2 if (arch == ffeq.PD and UP == 16) else 1)
        d_bytes = sum(p.n_sc * (p.C if arch == ffeq.FD else 1) * (p.U + p.n_sym) * p.U * 8 for p in ps)
        tables = 256 + len(ps) * (2 * 96 + 8 + 64 * 2)
        ws = ffeq.ffeq_batch_workspace_size(b)
        assert d_bytes + tables <= ws <= d_bytes + tables + 5 * 256


def test_instance_checks(lib):
    base = (64, 8, 4, 2, 3, 0.1, 1.0)

    def create(spec, **kw):
        cfg, inst = ffeq.pack_batch([spec], **kw)
        return ffeq.ffeq_batch_create(cfg, inst)

    assert _status(create, base) == 0
    assert _status(create, (64, 8, 3, 2, 3, 0.1, 1.0)) == 1          # B % C != 0
    assert _status(create, (64, 33, 4, 2, 3, 0.1, 1.0)) == 2         # U > 32
    assert _status(create, (64, 8, 4, 2, 17, 0.1, 1.0)) == 2         # n_sym > 16
    assert _status(create, (64, 8, 4, 2, 3, -0.1, 1.0)) == 1         # N0 < 0
    assert _status(create, (64, 8, 4, 2, 3, 0.1, 0.0)) == 1          # Es = 0
    assert _status(create, (64, 8, 4, 2, 3, float("inf"), 1.0)) == 1
    assert _status(create, (0, 8, 4, 2, 3, 0.1, 1.0)) == 1
    assert _status(create, (128, 8, 128, 1, 1, 0.1, 1.0), arch=ffeq.FD) == 2   # C * 8 > 512 lanes of one CTA
    # Offsets must lie inside the declared extents.
    cfg, inst = ffeq.pack_batch([base])
    inst[0].h_off = 2
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1
    cfg, inst = ffeq.pack_batch([base])
    inst[0].z_off = -2
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1
    cfg, inst = ffeq.pack_batch([base], llr_bits=4)
    cfg.llr_elems -= 1
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1
    cfg, inst = ffeq.pack_batch([base], arch=ffeq.FD)
    cfg.info_elems = 3                                               # needs n_sc * C = 8
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1
    cfg, inst = ffeq.pack_batch([base])
    cfg.arch = 5
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1


def test_empty_batch_needs_no_device(lib):
    cfg, inst = ffeq.pack_batch([])
    b = ffeq.ffeq_batch_create(cfg, inst)
    assert ffeq.ffeq_batch_groups(b) == 0
    assert ffeq.ffeq_batch_get_tuning(b) == []
    # Nothing to do: returns before any CUDA call (pointers are never touched).
    ffeq.ffeq_batch_equalize(b, 16, 16, 16, 16, None, None, 256, ffeq.ffeq_batch_workspace_size(b), stream=0)


def test_buffer_checks_precede_any_device_call(lib):
    cfg, inst = ffeq.pack_batch([(64, 8, 4, 2, 3, 0.1, 1.0)], llr_bits=4, with_info=False)
    b = ffeq.ffeq_batch_create(cfg, inst)
    nb = ffeq.ffeq_batch_workspace_size(b)
    ok = dict(H=256, y=256, z=256, sigma2=256, llr=256, info=None, workspace=256, workspace_bytes=nb)
    for bad in (dict(H=None), dict(z=8 + 4), dict(llr=None), dict(info=256), dict(workspace=512 + 16),
                dict(workspace_bytes=nb - 1)):
        args = {**ok, **bad}
        assert _status(ffeq.ffeq_batch_equalize, b, args["H"], args["y"], args["z"], args["sigma2"], args["llr"],
                       args["info"], args["workspace"], args["workspace_bytes"], stream=0) == 1, bad


def test_tuning_roundtrip_and_validation(lib):
    ps = synth.make_uneven(256, seed=3)
    cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.FD)
    b = ffeq.ffeq_batch_create(cfg, inst)
    tun = ffeq.ffeq_batch_get_tuning(b)
    ffeq.ffeq_batch_set_tuning(b, tun)
    assert ffeq.ffeq_batch_get_tuning(b) == tun
    UP, st, th, lpr = tun[0]
    for change in ((1, 0), (1, 4), (0, UP * 2 if UP < 32 else 8), (2, 96 + 1), (2, 1024), (3, 3)):
        t = [list(x) for x in tun]
        t[0][change[0]] = change[1]
        assert _status(ffeq.ffeq_batch_set_tuning, b, t) == 1, change
    assert _status(ffeq.ffeq_batch_set_tuning, b, tun[:-1]) == 1
    assert ffeq.ffeq_batch_get_tuning(b) == tun
    if UP == 32:
        t = [list(x) for x in tun]
        t[0][3] = 2                                                  # two lanes per row needs UP <= 16
        assert _status(ffeq.ffeq_batch_set_tuning, b, t) == 1


def test_equalizer_choice(lib):
    """ZF, MRC and LAMA batches plan like L-MMSE ones (MRC and LAMA: one lane per
    row); LAMA takes 1..64 iterations, the others none; an unknown equalizer is an
    argument error."""
    ps = synth.make_uneven(64, seed=5)
    for eq, iters, status in ((ffeq.LMMSE, 0, 0), (ffeq.ZF, 0, 0), (ffeq.MRC, 0, 0), (ffeq.LAMA, 6, 0),
                              (ffeq.LAMA, 0, 1), (ffeq.LAMA, 65, 1), (ffeq.ZF, 2, 1), (7, 0, 1), (-1, 0, 1)):
        cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.PD, llr_bits=4, equalizer=eq, lama_iters=iters)
        assert _status(ffeq.ffeq_batch_create, cfg, inst) == status, (eq, iters)
    cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.FD, llr_bits=4, equalizer=ffeq.LAMA, lama_iters=6)
    assert all(t[3] == 1 for t in ffeq.ffeq_batch_get_tuning(ffeq.ffeq_batch_create(cfg, inst)))
    # LAMA's prior is the LLR constellation, and its denoiser needs N0 > 0 in every instance.
    cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.FD, llr_bits=0, equalizer=ffeq.LAMA, lama_iters=6)
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1
    q = synth.make_problem(64, 4, 2, 2, 3, snr_db=10.0, bits=4, seed=2, noiseless=True)
    cfg, inst = ffeq.pack_batch(_specs(ps + [q]), arch=ffeq.FD, llr_bits=4, equalizer=ffeq.LAMA, lama_iters=6)
    assert _status(ffeq.ffeq_batch_create, cfg, inst) == 1
    cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.PD, llr_bits=4, equalizer=ffeq.MRC)
    b = ffeq.ffeq_batch_create(cfg, inst)
    tun = ffeq.ffeq_batch_get_tuning(b)
    assert all(t[3] == 1 for t in tun)
    for gi, (UP, st, th, lpr) in enumerate(tun):
        if UP <= 16:
            t = [list(x) for x in tun]
            t[gi][3] = 2                                    # MRC has no row sweep to split
            assert _status(ffeq.ffeq_batch_set_tuning, b, t) == 1


def test_tuning_cache_key_separates_equalizers(lib):
    """The cached launch shapes of a batch are keyed by everything the plan's
    groups and kernels depend on: the same shapes with another equalizer or
    iteration count take another entry."""
    from paper_1808_04473_gb300 import tuning
    ps = synth.make_uneven(32, seed=8)
    keys = {}
    for eq, iters in ((ffeq.LMMSE, 0), (ffeq.ZF, 0), (ffeq.MRC, 0), (ffeq.LAMA, 4), (ffeq.LAMA, 8)):
        cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.FD, llr_bits=4, equalizer=eq, lama_iters=iters)
        keys[(eq, iters)] = tuning.batch_key(ffeq.ffeq_batch_create(cfg, inst), "GPU")
    assert len(set(keys.values())) == len(keys)
    cfg, inst = ffeq.pack_batch(_specs(ps), arch=ffeq.FD, llr_bits=4)
    assert tuning.batch_key(ffeq.ffeq_batch_create(cfg, inst), "GPU") == keys[(ffeq.LMMSE, 0)]
