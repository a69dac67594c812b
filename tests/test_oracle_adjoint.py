"""Pins of the oracle's differentiable FD form and its adjoint (CPU).

The closed-form gradients are checked against central finite differences of
the forward map (the definition of the derivative) on tiny random problems, for
every argument: H, y, rho_c and nu.  The forward is pinned by the paper's FD
L-MMSE: with C = 1, rho = N0/Es and nu = 1 it is the literal PD estimate.
"""
import numpy as np
import pytest

from oracle import adjoint, lmmse
from paper_1808_04473_gb300 import synth


def _problem(seed=0, B=8, U=3, C=2, n_sc=2, n_sym=2):
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=5.0, bits=2, seed=seed)
    rng = np.random.default_rng(seed + 100)
    rho = rng.uniform(0.3, 1.2, C)
    nu = rng.uniform(0.2, 0.9, (C, U))
    H = p.H.astype(np.complex128)
    y = p.y.astype(np.complex128)
    return p, H, y, rho, nu


def _loss(z, s):
    return float(np.sum(np.abs(z - s) ** 2))


def test_forward_reduces_to_lmmse_for_one_cluster():
    p = synth.make_problem(16, 4, 1, 5, 3, seed=3)
    z, xs = adjoint.fd_train_forward(p.H, p.y, np.array([p.N0 / p.Es]), np.ones((1, 4)))
    ref = lmmse.equalize_pd(p.H, p.y, p.N0, p.Es, 1, "literal")
    np.testing.assert_allclose(z, ref["z"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(xs[:, 0], ref["z"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_finite_differences(seed):
    p, H, y, rho, nu = _problem(seed)
    s = p.s
    z, _ = adjoint.fd_train_forward(H, y, rho, nu)
    gz = 2.0 * (z - s)                                   # dL/dRe + i dL/dIm of sum |z - s|^2
    gH, gy, grho, gnu = adjoint.fd_train_backward(H, y, rho, nu, gz)

    fH = adjoint.finite_difference(lambda h: _loss(adjoint.fd_train_forward(h, y, rho, nu)[0], s), H)
    fy = adjoint.finite_difference(lambda t: _loss(adjoint.fd_train_forward(H, t, rho, nu)[0], s), y)
    fr = adjoint.finite_difference(lambda r: _loss(adjoint.fd_train_forward(H, y, r, nu)[0], s), rho)
    fn = adjoint.finite_difference(lambda w: _loss(adjoint.fd_train_forward(H, y, rho, w)[0], s), nu)
    for got, ref in ((gH, fH), (gy, fy), (grho, fr), (gnu, fn)):
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("sizes", [[2, 9, 5], [0, 7, 9]])
def test_unequal_clusters_match_finite_differences(sizes):
    """Clusters of given sizes (Sec. II-B; an empty one included): every gradient
    equals central differences of the forward on the same partition, and the
    forward's local estimates are each cluster's own L-MMSE solve."""
    p, H, y, rho, nu = _problem(7, B=16, U=3, C=3)
    s = p.s
    z, xs = adjoint.fd_train_forward(H, y, rho, nu, cluster_sizes=sizes)
    gz = 2.0 * (z - s)
    gH, gy, grho, gnu = adjoint.fd_train_backward(H, y, rho, nu, gz, cluster_sizes=sizes)

    def f(h, t, r, w):
        return _loss(adjoint.fd_train_forward(h, t, r, w, cluster_sizes=sizes)[0], s)

    fH = adjoint.finite_difference(lambda h: f(h, y, rho, nu), H)
    fy = adjoint.finite_difference(lambda t: f(H, t, rho, nu), y)
    fr = adjoint.finite_difference(lambda r: f(H, y, r, nu), rho)
    fn = adjoint.finite_difference(lambda w: f(H, y, rho, w), nu)
    for got, ref in ((gH, fH), (gy, fy), (grho, fr), (gnu, fn)):
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
    # Local estimates: the regularized least-squares solution of each cluster alone,
    # through an SVD (no normal equations), and zero for an empty cluster.
    b0 = 0
    for c, bc in enumerate(sizes):
        for k in range(H.shape[0]):
            Hc = H[k].T[b0:b0 + bc]
            Yc = y[k].T[b0:b0 + bc]
            A = np.vstack([Hc, np.sqrt(rho[c]) * np.eye(H.shape[1])])
            R = np.vstack([Yc, np.zeros((H.shape[1], Yc.shape[1]))])
            X = np.linalg.lstsq(A, R, rcond=None)[0]
            np.testing.assert_allclose(xs[k, c], X.T, rtol=1e-10, atol=1e-12)
        b0 += bc


def test_gradient_of_a_wrong_formula_is_caught():
    """Sanity of the pin itself: dropping the H G_b X^H term breaks the H gradient."""
    p, H, y, rho, nu = _problem(5)
    z, _ = adjoint.fd_train_forward(H, y, rho, nu)
    gz = 2.0 * (z - p.s)
    gH, *_ = adjoint.fd_train_backward(H, y, rho, nu, gz)
    fH = adjoint.finite_difference(lambda h: _loss(adjoint.fd_train_forward(h, y, rho, nu)[0], p.s), H)
    bounds = lmmse.partition(H.shape[2], len(rho))
    wrong = gH.copy()
    for k in range(H.shape[0]):
        for c, (b0, b1) in enumerate(bounds):
            Hc = H[k].T[b0:b1]
            M = Hc.conj().T @ Hc + rho[c] * np.eye(H.shape[1])
            X = np.linalg.solve(M, Hc.conj().T @ y[k].T[b0:b1])
            Gb = np.linalg.solve(M, nu[c][:, None] * gz[k].T)
            wrong[k, :, b0:b1] += (Hc @ (Gb @ X.conj().T)).T
    assert np.abs(wrong - fH).max() > 1e-3
    assert np.abs(gH - fH).max() < 1e-6 * max(1.0, np.abs(fH).max())


@pytest.mark.parametrize("seed,C,sizes", [(0, 2, None), (1, 3, [3, 5, 4]), (2, 1, None)])
def test_gradients_through_the_optimal_weights_match_finite_differences(seed, C, sizes):
    """FD with the unbiased pairs and Lemma 1's weights (the library's forward): the closed-form
    gradients with respect to H and y equal central differences of lmmse.equalize_fd."""
    B = 12
    p = synth.make_problem(B, 3, C, 2, 2, snr_db=5.0, bits=2, seed=seed)
    H, y = p.H.astype(np.complex128), p.y.astype(np.complex128)
    N0, Es = 0.6, 1.0

    def loss(h, t):
        return _loss(lmmse.equalize_fd(h, t, N0, Es, C, "unbiased", cluster_sizes=sizes)["z"], p.s)

    z = lmmse.equalize_fd(H, y, N0, Es, C, "unbiased", cluster_sizes=sizes)["z"]
    gH, gy = adjoint.fd_optimal_backward(H, y, N0, Es, C, 2.0 * (z - p.s), cluster_sizes=sizes)
    fH = adjoint.finite_difference(lambda h: loss(h, y), H)
    fy = adjoint.finite_difference(lambda t: loss(H, t), y)
    for got, ref in ((gH, fH), (gy, fy)):
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


def test_optimal_weight_term_is_needed():
    """Sanity of the pin: without the weights' dependence on diag(A_c) (the free-weight adjoint
    at the optimal weights) the H gradient misses the finite differences."""
    C = 2
    p = synth.make_problem(12, 3, C, 1, 2, snr_db=5.0, bits=2, seed=7)
    H, y = p.H.astype(np.complex128), p.y.astype(np.complex128)
    N0, Es = 0.6, 1.0
    rho = N0 / Es
    z = lmmse.equalize_fd(H, y, N0, Es, C, "unbiased")["z"]
    gz = 2.0 * (z - p.s)
    fH = adjoint.finite_difference(
        lambda h: _loss(lmmse.equalize_fd(h, y, N0, Es, C, "unbiased")["z"], p.s), H)
    # Frozen weights nu_c = w_c / D (the optimal ones at this point) through the free-weight adjoint.
    Hm = H[0].T
    ws = [1.0 / np.real(np.diag(np.linalg.inv(Hm[b0:b1].conj().T @ Hm[b0:b1] + rho * np.eye(3))))
          for b0, b1 in lmmse.partition(12, C)]
    D = sum(w - rho for w in ws)
    nu = np.array([w / D for w in ws])
    gH_frozen, *_ = adjoint.fd_train_backward(H, y, np.full(C, rho), nu, gz)
    gH, _ = adjoint.fd_optimal_backward(H, y, N0, Es, C, gz)
    assert np.abs(gH - fH).max() <= 1e-6 * max(1.0, np.abs(fH).max())
    assert np.abs(gH_frozen - fH).max() > 1e-3 * np.abs(fH).max()
