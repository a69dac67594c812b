"""GPU parity of the differentiable FD form and its hand-written adjoint.

Forward against ``oracle.adjoint.fd_train_forward`` (bound 1e-5 relative per
subcarrier and per entry, ``tests/parity.py``; FP32 arithmetic); backward against
the oracle's closed-form gradients, which are pinned by finite differences
(bound 1e-3, the stated target of the adjoint: per subcarrier and per entry for
dL/dH and dL/dy, relative to the largest entry for the gradients summed over
subcarriers, dL/drho and dL/dnu); and the autograd wrapper against the direct
C-ABI calls.
"""
import numpy as np
import pytest

import parity
from oracle import adjoint, lmmse
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


def _setup(B, U, C, n_sc, n_sym, seed, snr=10.0):
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=snr, bits=2, seed=seed)
    rng = np.random.default_rng(seed + 7)
    rho = (p.N0 / p.Es) * rng.uniform(0.5, 2.0, C)
    nu = rng.uniform(0.5, 1.5, (C, U)) / C
    return p, rho.astype(np.float32), nu.astype(np.float32)


def _run(ff, p, rho, nu, C, gz=None, sizes=None):
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    r = torch.from_numpy(rho).to(dev)
    w = torch.from_numpy(nu).to(dev)
    plan = ff.ffeq_plan_create(p.B, p.U, C, p.n_sc, p.n_sym, arch=ff.FD, cluster_sizes=sizes)
    nb = ff.ffeq_fd_train_workspace_size(plan)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    z = torch.empty((p.n_sc, p.n_sym, p.U), dtype=torch.complex64, device=dev)
    ff.ffeq_fd_train_forward(plan, H, y, r, w, z, ws, nb)
    out = {"z": z}
    if gz is not None:
        g = torch.from_numpy(gz.astype(np.complex64)).to(dev)
        out.update(gH=torch.empty_like(H), gy=torch.empty_like(y), grho=torch.empty_like(r), gnu=torch.empty_like(w))
        ff.ffeq_fd_train_backward(plan, H, y, r, w, g, out["gH"], out["gy"], out["grho"], out["gnu"], ws, nb)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("B,U,C,n_sc,n_sym", [(16, 3, 2, 7, 2), (64, 16, 4, 20, 3), (96, 12, 12, 5, 1),
                                              (128, 16, 8, 33, 1), (256, 32, 16, 6, 14)])
def test_forward_and_backward_match_the_oracle(ff, B, U, C, n_sc, n_sym):
    p, rho, nu = _setup(B, U, C, n_sc, n_sym, seed=B + U + C)
    z0, _ = adjoint.fd_train_forward(p.H, p.y, rho.astype(np.float64), nu.astype(np.float64))
    gz = 2.0 * (z0 - p.s) / z0.size                     # MSE loss
    g = _run(ff, p, rho, nu, C, gz)
    parity.check("z", g["z"], z0, 1e-5)
    gH, gy, grho, gnu = adjoint.fd_train_backward(p.H, p.y, rho.astype(np.float64), nu.astype(np.float64),
                                                  gz.astype(np.complex64).astype(np.complex128))
    parity.check("gH", g["gH"], gH, 1e-3)
    parity.check("gy", g["gy"], gy, 1e-3)
    for name, ref in (("grho", grho), ("gnu", gnu)):
        assert _relmax(g[name], ref) <= 1e-3, (name, _relmax(g[name], ref))


TRAIN_UNEQUAL = [  # B, U, C, n_sc, n_sym, sizes (Sec. II-B: clusters of given sizes)
    (20, 4, 3, 9, 2, [0, 13, 7]),            # an empty cluster; B % C != 0
    (96, 12, 3, 10, 5, [40, 24, 32]),
    (256, 32, 16, 5, 14, [8, 24, 16, 16, 12, 20, 16, 16, 16, 16, 10, 22, 16, 16, 16, 16]),
]


@pytest.mark.parametrize("B,U,C,n_sc,n_sym,sizes", TRAIN_UNEQUAL)
def test_unequal_clusters_match_the_oracle(ff, B, U, C, n_sc, n_sym, sizes):
    """The free-weight form on clusters of given sizes: forward and every gradient
    against the oracle on the same partition (bounds as for equal clusters)."""
    p = synth.make_problem(B, U, 1, n_sc, n_sym, snr_db=10.0, bits=2, seed=B + C)
    rng = np.random.default_rng(B + C + 7)
    rho = ((p.N0 / p.Es) * rng.uniform(0.5, 2.0, C)).astype(np.float32)
    nu = (rng.uniform(0.5, 1.5, (C, U)) / C).astype(np.float32)
    z0, _ = adjoint.fd_train_forward(p.H, p.y, rho.astype(np.float64), nu.astype(np.float64), cluster_sizes=sizes)
    gz = 2.0 * (z0 - p.s) / z0.size
    g = _run(ff, p, rho, nu, C, gz, sizes)
    parity.check("z", g["z"], z0, 1e-5)
    gH, gy, grho, gnu = adjoint.fd_train_backward(p.H, p.y, rho.astype(np.float64), nu.astype(np.float64),
                                                  gz.astype(np.complex64).astype(np.complex128), cluster_sizes=sizes)
    parity.check("gH", g["gH"], gH, 1e-3)
    parity.check("gy", g["gy"], gy, 1e-3)
    for name, ref in (("grho", grho), ("gnu", gnu)):
        assert _relmax(g[name], ref) <= 1e-3, (name, _relmax(g[name], ref))


def test_rho_and_nu_gradients_match_fp64_finite_differences(ff):
    """Direct check of the GPU gradients against central differences of the FP64 forward."""
    p, rho, nu = _setup(32, 4, 2, 6, 2, seed=3)
    r64, n64 = rho.astype(np.float64), nu.astype(np.float64)
    loss = lambda r, w: float(np.mean(np.abs(adjoint.fd_train_forward(p.H, p.y, r, w)[0] - p.s) ** 2))
    z0, _ = adjoint.fd_train_forward(p.H, p.y, r64, n64)
    g = _run(ff, p, rho, nu, 2, 2.0 * (z0 - p.s) / z0.size)
    fr = adjoint.finite_difference(lambda r: loss(r, n64), r64)
    fn = adjoint.finite_difference(lambda w: loss(r64, w), n64)
    assert _relmax(g["grho"], fr) <= 1e-3
    assert _relmax(g["gnu"], fn) <= 1e-3


def test_training_shaped_batch(ff):
    """B=128, U=16, C=8 (S=16), 1024 subcarriers x 8 channel draws, QPSK, 10 dB."""
    p, rho, nu = _setup(128, 16, 8, 8 * 1024, 1, seed=11)
    z0, _ = adjoint.fd_train_forward(p.H, p.y, rho.astype(np.float64), nu.astype(np.float64))
    gz = 2.0 * (z0 - p.s) / z0.size
    g = _run(ff, p, rho, nu, 8, gz)
    gH, gy, grho, gnu = adjoint.fd_train_backward(p.H, p.y, rho.astype(np.float64), nu.astype(np.float64),
                                                  gz.astype(np.complex64).astype(np.complex128))
    parity.check("z", g["z"], z0, 1e-5)
    parity.check("gH", g["gH"], gH, 1e-3)
    parity.check("gy", g["gy"], gy, 1e-3)
    for name, ref in (("grho", grho), ("gnu", gnu)):
        assert _relmax(g[name], ref) <= 1e-3, (name, _relmax(g[name], ref))


def test_autograd_function_matches_the_c_abi(ff):
    from paper_1808_04473_gb300.autograd import fd_equalize
    p, rho, nu = _setup(64, 8, 4, 16, 2, seed=21)
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev).requires_grad_(True)
    y = torch.from_numpy(p.y).to(dev).requires_grad_(True)
    r = torch.from_numpy(rho).to(dev).requires_grad_(True)
    w = torch.from_numpy(nu).to(dev).requires_grad_(True)
    s = torch.from_numpy(p.s.astype(np.complex64)).to(dev)
    z = fd_equalize(H, y, r, w, 4)
    loss = (z - s).abs().pow(2).mean()
    loss.backward()
    z0 = z.detach().cpu().numpy()
    gz = 2.0 * (z0 - p.s) / z0.size
    ref = _run(ff, p, rho, nu, 4, gz)
    for t, name in ((H, "gH"), (y, "gy"), (r, "grho"), (w, "gnu")):
        assert _relmax(t.grad.cpu().numpy(), ref[name]) <= 1e-5, name


# ---------------------------------------------------------------- gradients through the optimal weights

def _optimal(ff, p, C, gz, sizes=None, precision=0):
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    plan = ff.ffeq_plan_create(p.B, p.U, C, p.n_sc, p.n_sym, arch=ff.FD, precision=precision, cluster_sizes=sizes)
    nb = ff.ffeq_fd_optimal_workspace_size(plan)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    g = torch.from_numpy(gz.astype(np.complex64)).to(dev)
    gH, gy = torch.empty_like(H), torch.empty_like(y)
    ff.ffeq_fd_optimal_backward(plan, H, y, p.N0, p.Es, g, gH, gy, ws, nb)
    torch.cuda.synchronize()
    return gH.cpu().numpy(), gy.cpu().numpy()


OPT_CASES = [  # B, U, C, n_sc, n_sym, sizes
    (16, 3, 2, 7, 2, None),
    (64, 16, 4, 20, 3, None),
    (128, 8, 8, 24, 14, None),          # n_sym = 14 right-hand sides
    (96, 12, 3, 10, 5, [40, 24, 32]),   # clusters of given sizes (Sec. II-B)
    (100, 8, 3, 12, 2, [40, 35, 25]),   # B % C != 0
    (256, 32, 8, 4, 6, None),           # U = 32
]


@pytest.mark.parametrize("B,U,C,n_sc,n_sym,sizes", OPT_CASES)
def test_optimal_weight_adjoint_matches_the_oracle(ff, B, U, C, n_sc, n_sym, sizes):
    """dL/dH, dL/dy through Lemma 1's weights (ffeq_fd_optimal_backward) against the
    oracle's closed form (pinned to finite differences of the FD forward), 1e-3 per
    subcarrier and per entry, for an MSE loss of the FD estimate."""
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=8.0, bits=2, seed=B + 3 * U + C)
    N0 = float(np.float32(p.N0))
    z0 = lmmse.equalize_fd(p.H, p.y, N0, p.Es, C, "unbiased", cluster_sizes=sizes)["z"]
    gz = 2.0 * (z0 - p.s) / z0.size
    gH, gy = _optimal(ff, p, C, gz, sizes)
    oH, oy = adjoint.fd_optimal_backward(p.H, p.y, N0, p.Es, C, gz.astype(np.complex64).astype(np.complex128),
                                         cluster_sizes=sizes)
    parity.check("gH", gH, oH, 1e-3)
    parity.check("gy", gy, oy, 1e-3)
    assert ff.ffeq_device_status() == 0


def test_optimal_weight_adjoint_on_the_training_shape(ff):
    """B=128, U=16, C=8 (S=16), 8 x 1024 subcarriers, QPSK, 10 dB; 16 sampled subcarriers
    against the oracle (the GPU computes all of them)."""
    p = synth.make_problem(128, 16, 8, 8 * 1024, 1, snr_db=10.0, bits=2, seed=23)
    N0 = float(np.float32(p.N0))
    idx = np.random.default_rng(2).choice(p.n_sc, 16, replace=False)
    rng = np.random.default_rng(3)
    gz = (rng.standard_normal((p.n_sc, 1, 16)) + 1j * rng.standard_normal((p.n_sc, 1, 16))) / 8192.0
    gH, gy = _optimal(ff, p, 8, gz)
    oH, oy = adjoint.fd_optimal_backward(p.H[idx], p.y[idx], N0, p.Es, 8,
                                         gz[idx].astype(np.complex64).astype(np.complex128))
    parity.check("gH", gH[idx], oH, 1e-3)
    parity.check("gy", gy[idx], oy, 1e-3)
    assert np.isfinite(gH).all() and np.isfinite(gy).all()


def test_optimal_weight_adjoint_against_finite_differences(ff):
    """Directly against central differences of the FP64 FD forward (Lemma 1 weights)
    on a tiny case, for every entry of H and y."""
    p = synth.make_problem(12, 3, 2, 2, 2, snr_db=5.0, bits=2, seed=4)
    N0 = float(np.float32(p.N0))
    H, y = p.H.astype(np.complex128), p.y.astype(np.complex128)

    def loss(h, t):
        z = lmmse.equalize_fd(h, t, N0, p.Es, 2, "unbiased")["z"]
        return float(np.sum(np.abs(z - p.s) ** 2))

    z0 = lmmse.equalize_fd(H, y, N0, p.Es, 2, "unbiased")["z"]
    gH, gy = _optimal(ff, p, 2, 2.0 * (z0 - p.s))
    fH = adjoint.finite_difference(lambda h: loss(h, y), H)
    fy = adjoint.finite_difference(lambda t: loss(H, t), y)
    assert _relmax(gH, fH) <= 1e-3 and _relmax(gy, fy) <= 1e-3


def test_optimal_autograd_function_matches_the_c_abi(ff):
    from paper_1808_04473_gb300.autograd import fd_equalize_optimal
    p = synth.make_problem(64, 8, 4, 16, 2, snr_db=10.0, bits=2, seed=25)
    dev = torch.device("cuda:0")
    H = torch.from_numpy(p.H).to(dev).requires_grad_(True)
    y = torch.from_numpy(p.y).to(dev).requires_grad_(True)
    s = torch.from_numpy(p.s.astype(np.complex64)).to(dev)
    z = fd_equalize_optimal(H, y, p.N0, p.Es, 4)
    loss = (z - s).abs().pow(2).mean()
    loss.backward()
    z0 = z.detach().cpu().numpy()
    gz = 2.0 * (z0 - p.s) / z0.size
    gH, gy = _optimal(ff, p, 4, gz)
    assert _relmax(H.grad.cpu().numpy(), gH) <= 1e-5 and _relmax(y.grad.cpu().numpy(), gy) <= 1e-5
    # Its forward is the library's FD estimate.
    ref = ff.equalize(H.detach(), y.detach(), p.N0, p.Es, 4, arch=ff.FD)
    assert torch.equal(z.detach(), ref["z"])
