"""Pins of the learned corrector's oracle (``oracle/cnn.py``): bfloat16 rounding, the 3x3
convolution, the backward pass, Adam, the input features and the judged restart loop."""

import numpy as np
import pytest

import oracle
from oracle import cnn
from paper_1108_2045_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_bf16_rounding_values():
    one = 1.0
    ulp = 2.0 ** -7  # spacing of bfloat16 just above 1
    cases = [(one, one), (one + ulp / 2, one), (one + 3 * ulp / 2, one + 2 * ulp), (one + 0.75 * ulp, one + ulp),
             (-(one + 0.75 * ulp), -(one + ulp)), (0.0, 0.0), (3.0e38, 1.765625 * 2.0 ** 127), (1.0e-40, 2.0 ** -133)]
    for x, want in cases:
        assert cnn.bf16(x) == want, (x, cnn.bf16(x), want)
    assert np.isnan(cnn.bf16(np.nan))
    xs = np.random.default_rng(0).standard_normal(1000)
    got = cnn.bf16(xs)
    assert np.all(np.abs(got - xs) <= 2.0 ** -8 * np.abs(xs))  # unit roundoff of 8 significant bits
    for x in xs[:50]:  # the C oracle's rounding agrees
        assert cnn.bf16(x) == oracle.bf16_round(np.float32(x))


def test_conv_matches_scipy_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, 11, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    y = cnn.conv3x3(a, w)
    for o in range(4):
        ref = sum(signal.correlate2d(a[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_conv_of_a_delta_reproduces_the_kernel():
    w = np.arange(2 * 1 * 9, dtype=float).reshape(2, 1, 3, 3)
    a = np.zeros((1, 7, 7))
    a[0, 3, 3] = 1.0
    y = cnn.conv3x3(a, w)
    for p in range(3):
        for q in range(3):
            assert y[1, 3 - p + 1, 3 - q + 1] == w[1, 0, p, q]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = cnn.init_weights(3, c_in=2, width=4, layers=3)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    xs = [rng.standard_normal((2, 6, 5)) for _ in range(2)]
    ts = [rng.standard_normal((6, 5)) for _ in range(2)]
    loss, gw, gb = cnn.loss_and_grads(params, xs, ts, rounding=False)
    eps = 1e-6
    for l in range(3):
        w, b = params[l]
        for idx in [(0, 0, 0, 0), (0, 1, 2, 1), (w.shape[0] - 1, w.shape[1] - 1, 1, 2)]:
            wp = w.copy()
            wp[idx] += eps
            wm = w.copy()
            wm[idx] -= eps
            lp = cnn.loss_and_grads([(wp, b) if k == l else params[k] for k in range(3)], xs, ts, rounding=False)[0]
            lm = cnn.loss_and_grads([(wm, b) if k == l else params[k] for k in range(3)], xs, ts, rounding=False)[0]
            assert abs((lp - lm) / (2 * eps) - gw[l][idx]) <= 1e-6 * max(1.0, abs(gw[l][idx])), (l, idx)
        bp = b.copy()
        bp[0] += eps
        bm = b.copy()
        bm[0] -= eps
        lp = cnn.loss_and_grads([(w, bp) if k == l else params[k] for k in range(3)], xs, ts, rounding=False)[0]
        lm = cnn.loss_and_grads([(w, bm) if k == l else params[k] for k in range(3)], xs, ts, rounding=False)[0]
        assert abs((lp - lm) / (2 * eps) - gb[l][0]) <= 1e-6 * max(1.0, abs(gb[l][0]))


def test_adam_first_step_moves_by_the_learning_rate():
    # after one step m_hat = g and v_hat = g^2, so every weight moves by lr * sign(g)
    params = [(np.array([[[[0.5]]]]), np.array([0.25]))]
    gw = [np.array([[[[3.0]]]])]
    gb = [np.array([-0.02])]
    new, state = cnn.adam(params, gw, gb, None, 1, lr=1e-2)
    assert abs(new[0][0].item() - (0.5 - 1e-2)) < 1e-7 and abs(new[0][1].item() - (0.25 + 1e-2)) < 1e-7
    new2, _ = cnn.adam(new, gw, gb, state, 2, lr=1e-2)  # same gradient again: same step
    assert abs(new2[0][0].item() - (0.5 - 2e-2)) < 1e-6


def test_features_definitions():
    n = 32
    kc = inputs.grf_coefficient(n, ell=0.1, seed=4)
    f = inputs.normal_rhs(n, 2, seed=5)
    r = oracle.residual_vc(kc, f, np.zeros_like(f))
    x, rho = cnn.features(kc, r)
    assert x.shape == (2, n + 1, n + 1)
    assert abs(np.mean(x[0][1:-1, 1:-1] ** 2) - 1.0) < 1e-2  # unit RMS up to bfloat16 rounding
    assert np.all(x[0][0] == 0) and np.all(x[0][:, -1] == 0)
    np.testing.assert_allclose(x[1], np.log(kc), rtol=2.0 ** -8, atol=1e-6)
    # D(p) = 4 k for a constant coefficient; the residual of u = 0 is f
    D = cnn.diagonal(np.full((n + 1, n + 1), 2.5))
    assert np.all(D[1:-1, 1:-1] == 10.0) and np.all(D[0] == 0)
    assert abs(rho - np.sqrt(np.mean((f[1:-1, 1:-1] / (n * n) / cnn.diagonal(kc)[1:-1, 1:-1]) ** 2))) <= 1e-14 * rho


def test_zero_network_leaves_the_solver_unchanged():
    # a network that always proposes 0 is always rejected; the iterates are plain HOMG's
    n, levels = 32, 5
    kc = inputs.grf_coefficient(n, ell=0.1, seed=6)
    f = inputs.normal_rhs(n, 2, seed=7)
    params = [(np.zeros_like(w), np.zeros_like(b)) for w, b in cnn.init_weights(0, width=8)]
    u, st, cyc, hist, acc = cnn.solve_learned(kc, f, params, levels, tol=1e-10)
    u0, st0, cyc0, hist0 = oracle.solve_vc(kc, f, levels, tol=1e-10)
    assert (st, cyc) == (st0, cyc0) and not any(acc)
    np.testing.assert_array_equal(u, u0)


def test_learned_solve_reaches_tolerance_with_a_random_network():
    n, levels = 32, 5
    kc = inputs.grf_coefficient(n, ell=0.1, seed=8)
    f = inputs.normal_rhs(n, 2, seed=9)
    params = cnn.init_weights(1, width=8)
    u, st, cyc, hist, acc = cnn.solve_learned(kc, f, params, levels, tol=1e-10)
    assert st == oracle.OK and hist[-1] <= 1e-10
    assert oracle.norm_interior(oracle.residual_vc(kc, f, u)) / oracle.norm_interior(f) <= 1e-10


def jacobi_network(c, width=32):
    """A network whose output is exactly c x_0: the first layer splits x_0 into relu(x_0) and
    relu(-x_0), two identity layers carry them, the last layer forms c (relu(x_0) - relu(-x_0)).
    Its proposal u + rho c x_0 = u + c h^2 r / D is one damped-Jacobi step of weight c."""
    shapes = cnn.shapes(width=width)
    params = [(np.zeros((co, ci, 3, 3)), np.zeros(co)) for co, ci in shapes]
    params[0][0][0, 0, 1, 1] = 1.0
    params[0][0][1, 0, 1, 1] = -1.0
    for l in (1, 2):
        params[l][0][0, 0, 1, 1] = 1.0
        params[l][0][1, 1, 1, 1] = 1.0
    params[3][0][0, 0, 1, 1] = c
    params[3][0][0, 1, 1, 1] = -c
    return params


def test_jacobi_network_output_is_exact():
    rng = np.random.default_rng(20)
    x = cnn.bf16(rng.standard_normal((2, 9, 11)))
    y, _ = cnn.forward(jacobi_network(0.75), x)
    np.testing.assert_array_equal(y, 0.75 * x[0])


def test_residual_loss_vanishes_for_the_exact_local_correction():
    # when x_0 is exactly the scaled operator applied to y, the proposal y removes the whole
    # residual at every inner pixel: the loss is 0 (up to rounding)
    rng = np.random.default_rng(21)
    x = np.stack([np.zeros((7, 8)), rng.uniform(-1.0, 1.0, (7, 8))])
    y = rng.standard_normal((7, 8))
    w = cnn.patch_operator(x)
    nb = [y[1:-1, :-2], y[1:-1, 2:], y[:-2, 1:-1], y[2:, 1:-1]]
    x[0, 1:-1, 1:-1] = y[1:-1, 1:-1] - sum(wq * q for wq, q in zip(w, nb))
    res, _ = cnn.residual_loss_terms(x, y)
    assert np.max(np.abs(res)) <= 1e-14
    # constant coefficient: every weight is 1/4, the scaled operator is y - mean of the 4 neighbours
    xc = np.stack([np.zeros((5, 5)), np.full((5, 5), 0.3)])
    assert np.allclose(cnn.patch_operator(xc), 0.25, rtol=0, atol=1e-15)


def test_residual_loss_gradients_match_finite_differences():
    rng = np.random.default_rng(22)
    params = cnn.init_weights(5, c_in=2, width=4, layers=3)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    xs = [np.stack([rng.standard_normal((6, 7)), rng.uniform(-1, 1, (6, 7))]) for _ in range(2)]
    ts = [np.zeros((6, 7))] * 2
    loss, gw, gb = cnn.loss_and_grads(params, xs, ts, rounding=False, loss_kind="residual")
    # a constant added to the output changes no residual (the weights w_q(p) sum to 1): the last
    # bias has gradient 0
    assert np.abs(gb[-1]).max() <= 1e-12 * np.abs(gw[-1]).max()
    eps = 1e-6
    for l in range(3):
        w, b = params[l]
        for idx in [(0, 0, 0, 0), (0, 1, 2, 1), (w.shape[0] - 1, w.shape[1] - 1, 1, 2)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            lp = cnn.loss_and_grads([(wp, b) if k == l else params[k] for k in range(3)], xs, ts, rounding=False,
                                    loss_kind="residual")[0]
            lm = cnn.loss_and_grads([(wm, b) if k == l else params[k] for k in range(3)], xs, ts, rounding=False,
                                    loss_kind="residual")[0]
            assert abs((lp - lm) / (2 * eps) - gw[l][idx]) <= 1e-6 * max(1.0, abs(gw[l][idx])), (l, idx)


@pytest.mark.parametrize("judge", ["proposal", "after_cycle"])
def test_zero_network_is_plain_homg_under_both_judges(judge):
    # a zero proposal never wins (equal residuals), so after two rejections the solve is plain HOMG
    n, levels = 32, 5
    kc = inputs.grf_coefficient(n, ell=0.1, seed=23)
    f = inputs.normal_rhs(n, 2, seed=24)
    params = [(np.zeros_like(w), np.zeros_like(b)) for w, b in cnn.init_weights(0, width=8)]
    u, st, cyc, hist, acc = cnn.solve_learned(kc, f, params, levels, tol=1e-10, judge=judge)
    u0, st0, cyc0, hist0 = oracle.solve_vc(kc, f, levels, tol=1e-10)
    assert (st, cyc) == (st0, cyc0) and acc == [False] * cyc
    np.testing.assert_array_equal(u, u0)


def test_jacobi_proposals_are_kept_and_an_amplifier_is_dropped_after_two_rejections():
    # constant coefficient: a damped-Jacobi step (weight 3/4) strictly lowers the residual norm, so the
    # judge keeps it; a step of weight -1 raises it, is rejected twice and then no longer proposed
    n, levels = 32, 5
    kc = np.full((n + 1, n + 1), 1.7)
    f = inputs.normal_rhs(n, 2, seed=25)
    _, st, cyc, _, acc = cnn.solve_learned(kc, f, jacobi_network(0.75, width=8), levels, tol=1e-10, max_cycles=3)
    assert acc[0] is True
    _, st, cyc, _, acc = cnn.solve_learned(kc, f, jacobi_network(-1.0, width=8), levels, tol=1e-10, max_cycles=4)
    assert acc == [False, False, False, False]
    # judged after the cycle, the proposal's result wins exactly when its residual after the cycle is lower
    u, st, cyc, hist, acc = cnn.solve_learned(kc, f, jacobi_network(0.75, width=8), levels, tol=0.0, max_cycles=1,
                                              judge="after_cycle")
    x, rho = cnn.features(kc, oracle.residual_vc(kc, f, np.zeros_like(f)))
    up = oracle.cycle_vc(kc, oracle.residual_vc(kc, f, np.zeros_like(f)), levels)
    u2 = np.zeros_like(f)
    u2[1:-1, 1:-1] = rho * 0.75 * x[0][1:-1, 1:-1]
    uq = u2 + oracle.cycle_vc(kc, oracle.residual_vc(kc, f, u2), levels)
    better = oracle.norm_interior(oracle.residual_vc(kc, f, uq)) < oracle.norm_interior(oracle.residual_vc(kc, f, up))
    assert acc == [better]
    np.testing.assert_array_equal(u, uq if better else up)
