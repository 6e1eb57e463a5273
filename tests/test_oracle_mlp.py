"""Pins of the FP64 warm-start network reference (CPU): its gradient against central finite
differences of its loss, invariants of a network with zero hidden weights, gradient descent on
a network without hidden layers reaching the least-squares solution of numpy.linalg.lstsq,
and the targets / features on cases with known values."""
import numpy as np

from oracle import mlp_oracle as MO
from oracle import KB_EVK


def _case(seed=3, n=20, width=8, depth=3):
    rng = np.random.default_rng(seed)
    params = MO.init_params(MO.NFEAT, width, depth, MO.NOUT, seed)
    params = [(W, rng.normal(0, 0.3, size=b.shape)) for W, b in params]   # nonzero biases too
    x = rng.normal(size=(n, MO.NFEAT))
    t = rng.normal(size=(n, MO.NOUT))
    return params, x, t


def test_gradient_matches_central_differences():
    params, x, t = _case()
    g = MO.flatten([(dW, db) for dW, db in MO.gradients(params, x, t)])
    v = MO.flatten(params)
    h = 1e-6
    fd = np.empty_like(v)
    for i in range(len(v)):
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd[i] = (MO.loss(MO.unflatten(vp, params), x, t) - MO.loss(MO.unflatten(vm, params), x, t)) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_zero_hidden_weights():
    """With every hidden weight zero the hidden states are constant, so the first layers get
    no weight gradient and the output bias gradient is the mean residual."""
    params, x, t = _case()
    params = [(np.zeros_like(W) if l < len(params) - 1 else W, b) for l, (W, b) in enumerate(params)]
    grads = MO.gradients(params, x, t)
    y, _ = MO.forward(params, x)
    for l in range(len(params) - 2):
        assert np.all(grads[l][0] == 0.0)
    np.testing.assert_allclose(grads[-1][1], (y - t).mean(axis=0), rtol=1e-12, atol=1e-14)


def test_linear_network_descends_to_least_squares():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(64, MO.NFEAT))
    t = rng.normal(size=(64, MO.NOUT))
    params = MO.init_params(MO.NFEAT, 1, 0, MO.NOUT, 7)     # no hidden layer: y = W x + b
    for _ in range(4000):
        (dW, db), = MO.gradients(params, x, t)
        (W, b), = params
        params = [(W - 0.5 * dW, b - 0.5 * db)]
    A = np.hstack([x, np.ones((len(x), 1))])
    sol = np.linalg.lstsq(A, t, rcond=None)[0]
    (W, b), = params
    np.testing.assert_allclose(W, sol[:-1].T, atol=1e-8)
    np.testing.assert_allclose(b, sol[-1], atol=1e-8)


def test_targets_and_features():
    rng = np.random.default_rng(2)
    T, mu = 300.0, 0.05
    eps = rng.uniform(-0.2, 0.2, size=10)
    x = (eps - mu) / (KB_EVK * T)
    v = rng.normal(size=(10, 3))
    v[3] = 0.0
    W = rng.uniform(1e12, 1e13, size=10)
    J0 = v / W[:, None]
    I0 = ((eps - mu) / T)[:, None] * J0
    speed = np.linalg.norm(v, axis=1)
    np.testing.assert_allclose(MO.scale_targets(I0, J0, J0, x, speed), 0.0, atol=1e-9)
    a = MO.scale_targets(I0 + 0.5 * KB_EVK * J0, 2.0 * J0, J0, x, speed)
    assert np.all(a[3] == 0.0)
    np.testing.assert_allclose(np.delete(a[:, 0], 3), 0.5, rtol=1e-9)
    np.testing.assert_allclose(np.delete(a[:, 1], 3), 1.0, rtol=1e-12)
    Iw, Jw = MO.warm_start(I0, J0, a)
    np.testing.assert_allclose(Iw, I0 + 0.5 * KB_EVK * J0, rtol=1e-9, atol=1e-30)
    np.testing.assert_allclose(Jw, 2.0 * J0, rtol=1e-12)
    f = MO.state_features(np.array([0.1, -0.2]), np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 1.0]]),
                          np.array([1e13, 0.0]), 300.0, 0.05)
    np.testing.assert_allclose(f[:, 0], np.array([0.05, -0.25]) / (KB_EVK * 300.0) / 10.0, rtol=1e-15)
    np.testing.assert_allclose(f[:, 1], [0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(f[:, 2], [1.0, 0.2], rtol=1e-15)
    np.testing.assert_allclose(f[:, 3:], [[1.0, 0.5, 1.0 / 3.0], [1.0, 0.5, -2.0 / 3.0]], rtol=1e-15)


def test_starting_responses_leave_the_answer_unchanged():
    """The coupled iteration is a contraction: any start reaches the same coefficients, and a
    start at the converged responses stops after its first outer check."""
    from oracle import prepare, transition_rates, solve_coupled_bte, TENSORS
    from paper_2109_08547_gb300 import synthetic as SY
    wl = SY.workload_sc1(n=6)
    P = prepare(wl)
    R = transition_rates(P)
    ref = solve_coupled_bte(P, R, level="dragged")
    odd = solve_coupled_bte(P, R, level="dragged", init=(1.3 * ref.I0, 0.8 * ref.J0))
    for key in TENSORS:
        a, b = odd.coeffs[key], ref.coeffs[key]
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b), key
    again = solve_coupled_bte(P, R, level="dragged", init=(ref.I, ref.J))
    assert again.converged and again.outer_iters <= 2 < ref.outer_iters
