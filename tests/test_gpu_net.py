"""Learned corrector on the GPU (tcgen05 convolutions, training kernels, features, judged solve) vs
the oracle in ``oracle/cnn.py`` (GB300 only).

Bars: an integer-valued network whose every intermediate value is exactly representable must come
out bit-exact (this pins the tensor-core operand layouts); random networks within bfloat16-storage
tolerances (relative L2 1e-2); gradients within 3e-2 per layer; features within one bfloat16 unit;
the zero network must leave the solver's iterates bit-identical to plain HOMG.
"""

import numpy as np
import pytest

import oracle
from oracle import cnn
from paper_1108_2045_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def homg():
    import torch

    import __graft_entry__

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    oracle.build()
    from paper_1108_2045_gb300 import homg as binding

    return binding


def flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


def unflat(v):
    out, off = [], 0
    for co, ci in cnn.shapes():
        nw = co * ci * 9
        out.append((v[off:off + nw].reshape(co, ci, 3, 3).astype(np.float64), v[off + nw:off + nw + co].astype(np.float64)))
        off += nw + co
    return out


def to_device_images(homg, xs):
    """list of [2, H, W] float arrays (bfloat16 values) -> device bfloat16 tensor [B, H, 2, W, 8]."""
    import torch

    arr = np.stack([homg.image_channels_first_to_device_layout(x.astype(np.float32)) for x in xs])
    return torch.from_numpy(arr).to(torch.bfloat16).cuda()


def gpu_forward(homg, params, xs, rows=None):
    import torch

    x = to_device_images(homg, xs)
    B, H, _, W, _ = x.shape
    y = torch.empty(B, H, W, dtype=torch.float32, device="cuda")
    with homg.Net() as net:
        if rows is not None:
            net.set_tile_rows(rows)
        net.set_params(flat(params))
        net.forward(x, y)
    return y.cpu().numpy().astype(np.float64)


def integer_network(seed):
    rng = np.random.default_rng(seed)
    nnz = [3, 4, 4, 6]
    params = []
    for l, (co, ci) in enumerate(cnn.shapes()):
        w = np.zeros((co, ci, 3, 3))
        for o in range(co):
            idx = rng.choice(ci * 9, size=nnz[l], replace=False)
            w[o].reshape(-1)[idx] = rng.choice([-1.0, 1.0], size=nnz[l])
        params.append((w, rng.integers(-1, 2, size=co).astype(np.float64)))
    return params


@pytest.mark.parametrize("rows", [4, 8])
def test_integer_network_is_exact(homg, rows):
    # B = 2 images of 37 x 150 pixels: two tiles across, a ragged last row band (for tiles of 4 and
    # of 8 output rows)
    rng = np.random.default_rng(1)
    params = integer_network(2)
    xs = [rng.integers(-2, 3, size=(2, 37, 150)).astype(np.float64) for _ in range(2)]
    for x in xs:  # every activation is an integer of magnitude <= 256: exact in bfloat16
        _, acts = cnn.forward(params, x)
        for a in acts[1:]:
            assert np.all(a == np.round(a)) and np.abs(a).max() <= 256
    ref = np.stack([cnn.forward(params, x)[0] for x in xs])
    got = gpu_forward(homg, params, xs, rows)
    np.testing.assert_array_equal(got, ref)


def test_tile_rows_do_not_change_the_result(homg):
    # every output row accumulates its products in the same order (vertical taps 0, 1, 2, then column
    # taps, then channel groups) whatever the tile height: bit-identical outputs
    rng = np.random.default_rng(40)
    params = [(w, cnn.f32(rng.standard_normal(b.shape) * 0.1)) for w, b in cnn.init_weights(41)]
    xs = [cnn.bf16(rng.standard_normal((2, 29, 300))) for _ in range(3)]
    np.testing.assert_array_equal(gpu_forward(homg, params, xs, 4), gpu_forward(homg, params, xs, 8))
    with homg.Net() as net:
        with pytest.raises(homg.HomgError):
            net.set_tile_rows(6)


@pytest.mark.parametrize("H,W", [(20, 130), (9, 64), (5, 7)])
def test_random_network_matches_oracle(homg, H, W):
    rng = np.random.default_rng(H * 1000 + W)
    params = [(w, cnn.f32(rng.standard_normal(b.shape) * 0.1)) for w, b in cnn.init_weights(3)]
    params[-1] = (params[-1][0] * 10.0, params[-1][1])
    xs = [cnn.bf16(rng.standard_normal((2, H, W))) for _ in range(2)]
    ref = np.stack([cnn.forward(params, x)[0] for x in xs])
    got = gpu_forward(homg, params, xs)
    assert np.linalg.norm(got - ref) <= 1e-2 * np.linalg.norm(ref)
    assert np.mean(np.abs(got - ref) <= 2e-2 * np.abs(ref).max()) >= 0.99


@pytest.mark.parametrize("rows", [4, 8])
def test_train_step_gradients_match_oracle(homg, rows):
    import torch

    rng = np.random.default_rng(5)
    params = [(w, cnn.f32(rng.standard_normal(b.shape) * 0.05)) for w, b in cnn.init_weights(4)]
    params[-1] = (params[-1][0] * 10.0, params[-1][1])
    B, P = 3, 64
    xs = [cnn.bf16(rng.standard_normal((2, P, P))) for _ in range(B)]
    ts = [cnn.f32(rng.standard_normal((P, P))) for _ in range(B)]
    loss_ref, gw, gb = cnn.loss_and_grads(params, xs, ts)
    x = to_device_images(homg, xs)
    t = torch.from_numpy(np.stack(ts).astype(np.float32)).cuda()
    lr = 1e-3
    with homg.Net() as net:
        net.set_tile_rows(rows)
        net.set_params(flat(params))
        loss = net.train_step(x, t, lr)
        grads = unflat(net.get_grads())
        after = net.get_params()
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    for l in range(len(params)):
        gW, gB = grads[l]
        assert np.linalg.norm(gW - gw[l]) <= 3e-2 * np.linalg.norm(gw[l]), l
        assert np.linalg.norm(gB - gb[l]) <= 3e-2 * np.linalg.norm(gb[l]) + 1e-12, l
    # Adam's first step moves every parameter by about lr * sign(g)
    step = after - flat(params)
    assert np.abs(step).max() <= lr * 1.001
    g_ref = np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in zip(gw, gb)])
    big = np.abs(g_ref) > 1e-2 * np.abs(g_ref).max()
    assert np.mean(np.sign(step[big]) == -np.sign(g_ref[big])) >= 0.98


def test_training_reduces_the_loss(homg):
    import torch

    rng = np.random.default_rng(6)
    B, P = 8, 64
    xs = [cnn.bf16(rng.standard_normal((2, P, P))) for _ in range(B)]
    kern = np.array([[[[0.1, 0.2, 0.1], [0.2, 0.4, 0.2], [0.1, 0.2, 0.1]]]])
    ts = [cnn.f32(cnn.conv3x3(x[:1], kern)[0]) for x in xs]  # a smoothing of channel 0: learnable
    x = to_device_images(homg, xs)
    t = torch.from_numpy(np.stack(ts).astype(np.float32)).cuda()
    with homg.Net() as net:
        net.set_params(flat(cnn.init_weights(7)))
        losses = [net.train_step(x, t, 3e-3) for _ in range(80)]
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def test_features_match_oracle(homg):
    import torch

    n = 64
    kc = inputs.grf_coefficient(n, ell=0.1, seed=8)
    f_np = inputs.normal_rhs(n, 2, seed=9)
    u_np = 1e-3 * inputs.normal_rhs(n, 2, seed=10)
    uref_np = 1e-3 * inputs.normal_rhs(n, 2, seed=11)
    f, u, uref = (torch.from_numpy(a).cuda() for a in (f_np, u_np, uref_np))
    x = torch.zeros(1, n + 1, 2, n + 1, 8, dtype=torch.bfloat16, device="cuda")
    t = torch.zeros(n + 1, n + 1, dtype=torch.float32, device="cuda")
    with homg.Solver(2, n + 1, 6) as s:
        s.set_coefficient(torch.from_numpy(kc).cuda())
        rho = homg.homg_features(s.handle, f, u, x, u_ref=uref, t_out=t)
    xr, rho_ref = cnn.features(kc, oracle.residual_vc(kc, f_np, u_np))
    assert abs(rho - rho_ref) <= 1e-12 * rho_ref
    got = homg.image_device_layout_to_channels_first(x[0].float().cpu().numpy())
    assert np.all(got[2:] == 0)
    for c in range(2):
        ulp = 2.0 ** -7 * np.abs(xr[c])
        assert np.all(np.abs(got[c] - xr[c]) <= ulp + 1e-30), c
        assert np.mean(got[c] == xr[c]) >= 0.999
    tref = np.zeros_like(f_np)
    tref[1:-1, 1:-1] = (uref_np - u_np)[1:-1, 1:-1] / rho_ref
    np.testing.assert_allclose(t.cpu().numpy(), tref, rtol=1e-6, atol=1e-6 * np.abs(tref).max())


def test_gather_patches(homg):
    import torch

    H, W, P = 40, 50, 16
    rng = np.random.default_rng(12)
    xs = cnn.bf16(rng.standard_normal((2, H, W)))
    x = to_device_images(homg, [xs])
    tn = rng.standard_normal((H, W)).astype(np.float32)
    t = torch.from_numpy(tn).cuda()
    corners_np = np.array([[0, 0], [H - P, W - P], [7, 11]], dtype=np.int32)
    corners = torch.from_numpy(corners_np).cuda()
    xp = torch.zeros(3, P, 2, P, 8, dtype=torch.bfloat16, device="cuda")
    tp = torch.zeros(3, P, P, dtype=torch.float32, device="cuda")
    with homg.Net() as net:
        net.gather_patches(x, t, corners, P, xp, tp)
        torch.cuda.synchronize()
    for b, (r0, c0) in enumerate(corners_np):
        got = homg.image_device_layout_to_channels_first(xp[b].float().cpu().numpy())
        np.testing.assert_array_equal(got[:2], xs[:, r0:r0 + P, c0:c0 + P])
        np.testing.assert_array_equal(tp[b].cpu().numpy(), tn[r0:r0 + P, c0:c0 + P])


def vc_problem(n, seed):
    return inputs.grf_coefficient(n, ell=0.1, seed=seed), inputs.normal_rhs(n, 2, seed=seed + 1)


def test_zero_network_learned_solve_is_plain_homg(homg):
    import torch

    n, levels = 128, 7
    kc, f_np = vc_problem(n, 13)
    f = torch.from_numpy(f_np).cuda()
    with homg.Solver(2, n + 1, levels) as s, homg.Net() as net:
        s.set_coefficient(torch.from_numpy(kc).cuda())
        u0 = torch.zeros_like(f)
        st0, c0, r0 = s.solve(f, u0, tol=1e-10, max_cycles=60)
        u1 = torch.zeros_like(f)
        st1, c1, r1, acc = homg.homg_solve_learned(s.handle, net, f, u1, tol=1e-10, max_cycles=60)
    assert (st1, c1, r1) == (st0, c0, r0) and not any(acc)
    assert torch.equal(u0, u1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_learned_solve_converges(homg, precision):
    import torch

    n, levels = 256, 8
    kc, f_np = vc_problem(n, 14)
    f = torch.from_numpy(f_np).cuda()
    params = cnn.init_weights(15)
    with homg.Solver(2, n + 1, levels, precision=precision) as s, homg.Net() as net:
        s.set_coefficient(torch.from_numpy(kc).cuda())
        net.set_params(flat(params))
        u = torch.zeros_like(f)
        st, cyc, rr, acc = homg.homg_solve_learned(s.handle, net, f, u, tol=1e-10, max_cycles=80)
    assert st == homg.HOMG_OK and rr <= 1e-10 and len(acc) == cyc
    got = u.cpu().numpy()
    assert oracle.norm_interior(oracle.residual_vc(kc, f_np, got)) / oracle.norm_interior(f_np) <= 1.0001e-10


def test_full_size_network_sampled_against_oracle(homg):
    # the 2049^2 variable-coefficient workload's first network input (u = 0), the network on the whole
    # image, checked at sampled pixels against the oracle on 9 x 9 crops
    import torch

    n = 2048
    kc = inputs.grf_coefficient(n, sigma=1.0, ell=0.05, seed=2)
    f_np = inputs.normal_rhs(n, 2, seed=0)
    rng = np.random.default_rng(16)
    params = [(w, cnn.f32(rng.standard_normal(b.shape) * 0.1)) for w, b in cnn.init_weights(17)]
    f = torch.from_numpy(f_np).cuda()
    u = torch.zeros_like(f)
    x = torch.zeros(1, n + 1, 2, n + 1, 8, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(1, n + 1, n + 1, dtype=torch.float32, device="cuda")
    with homg.Solver(2, n + 1, 11) as s, homg.Net() as net:
        s.set_coefficient(torch.from_numpy(kc).cuda())
        homg.homg_features(s.handle, f, u, x)
        net.set_params(flat(params))
        net.forward(x, y)
    ximg = homg.image_device_layout_to_channels_first(x[0].float().cpu().numpy())[:2].astype(np.float64)
    yg = y[0].cpu().numpy()
    # pixels at least 4 from the border, so a 9 x 9 crop holds the whole receptive field and no
    # hidden activation outside the image (the image borders are covered by the small-image tests)
    pts = [(4, 4), (4, n - 4), (n - 4, 4), (n - 4, n - 4), (4, 1000), (n - 4, 77), (1500, n - 5)]
    pts += [tuple(p) for p in rng.integers(4, n - 3, size=(24, 2))]
    for (py, px) in pts:
        crop = ximg[:, py - 4:py + 5, px - 4:px + 5]
        ref = cnn.forward(params, crop)[0][4, 4]
        assert abs(yg[py, px] - ref) <= 2e-2 * max(1.0, abs(ref)), (py, px, yg[py, px], ref)


def test_barrier_wait_gives_up_and_context_stays_usable(homg):
    # a convolution whose completion barrier nothing signals: the bounded wait must return an error
    # status (after 0.5 s, not hang), and the same network must work normally afterwards
    rng = np.random.default_rng(18)
    params = integer_network(19)
    xs = [rng.integers(-2, 3, size=(2, 9, 20)).astype(np.float64)]
    with homg.Net() as net:
        rc, ms = net.check_barrier_timeout()
        assert rc == homg.HOMG_ECUDA and "timed out" in homg.homg_net_last_error(net.handle)
        assert 400.0 <= ms <= 5000.0, ms
    ref = np.stack([cnn.forward(params, x)[0] for x in xs])
    np.testing.assert_array_equal(gpu_forward(homg, params, xs), ref)


def test_residual_loss_train_step_matches_oracle(homg):
    """The residual loss (homg_net_set_loss) against oracle/cnn.py's residual loss and its gradients,
    on patches whose log k channel varies (so the rebuilt operator's weights are not all 1/4)."""
    import torch

    rng = np.random.default_rng(30)
    params = [(w, cnn.f32(rng.standard_normal(b.shape) * 0.05)) for w, b in cnn.init_weights(31)]
    params[-1] = (params[-1][0] * 10.0, params[-1][1])
    B, P = 3, 64
    xs = [np.stack([cnn.bf16(rng.standard_normal((P, P))), cnn.bf16(rng.uniform(-2.0, 2.0, (P, P)))]) for _ in range(B)]
    ts = [np.zeros((P, P))] * B
    loss_ref, gw, gb = cnn.loss_and_grads(params, xs, ts, loss_kind="residual")
    x = to_device_images(homg, xs)
    t = torch.zeros(B, P, P, dtype=torch.float32, device="cuda")
    with homg.Net() as net:
        net.set_params(flat(params))
        net.set_loss("residual")
        loss = net.train_step(x, t, 1e-3)
        grads = unflat(net.get_grads())
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref, (loss, loss_ref)
    for l in range(len(params)):
        gW, gB = grads[l]
        assert np.linalg.norm(gW - gw[l]) <= 3e-2 * np.linalg.norm(gw[l]), l
        if l < len(params) - 1:
            assert np.linalg.norm(gB - gb[l]) <= 3e-2 * np.linalg.norm(gb[l]) + 1e-12, l
        else:
            # the last bias's gradient is exactly 0 (the weights w_q(p) sum to 1, so a constant shift
            # of the output leaves every residual unchanged): only rounding of the bfloat16 gradient
            # image remains, judged against the layer's weight gradient
            assert np.linalg.norm(gb[l]) <= 1e-12 * np.linalg.norm(gw[l])
            assert np.linalg.norm(gB) <= 1e-2 * np.linalg.norm(gw[l]), (gB, np.linalg.norm(gw[l]))


def jacobi_network(c):
    """Output exactly c x_0 (see tests/test_oracle_cnn.py): the proposal is a damped-Jacobi step."""
    params = [(np.zeros((co, ci, 3, 3)), np.zeros(co)) for co, ci in cnn.shapes()]
    params[0][0][0, 0, 1, 1] = 1.0
    params[0][0][1, 0, 1, 1] = -1.0
    for l in (1, 2):
        params[l][0][0, 0, 1, 1] = 1.0
        params[l][0][1, 1, 1, 1] = 1.0
    params[3][0][0, 0, 1, 1] = c
    params[3][0][0, 1, 1, 1] = -c
    return params


# Iterates of the learned loop against the oracle's: the network input is a bfloat16 rounding of the
# scaled FP64 residual, and the GPU's residual (another summation order) rounds to a neighbouring
# bfloat16 value at a few nodes, so the proposals differ there by one bfloat16 unit (2^-8 relative).
LEARNED_ITERATE_TOL = 2e-2


@pytest.mark.parametrize("judge", ["proposal", "after_cycle"])
@pytest.mark.parametrize("c", [0.75, -1.0])
def test_learned_loop_matches_oracle(homg, judge, c):
    """homg_solve_learned with a fixed non-zero network (a damped-Jacobi step of weight c: 0.75 is
    kept by the judge, -1 is rejected and then dropped) gives the oracle's keep/reject sequence and
    iterates within LEARNED_ITERATE_TOL after every cycle, under both judges."""
    import torch

    n, levels = 128, 7
    kc = inputs.grf_coefficient(n, ell=0.1, seed=32)
    f_np = inputs.normal_rhs(n, 2, seed=33)
    params = jacobi_network(c)
    f = torch.from_numpy(f_np).cuda()
    with homg.Solver(2, n + 1, levels) as s, homg.Net() as net:
        s.set_coefficient(torch.from_numpy(kc).cuda())
        homg.homg_set_learned_judge(s.handle, judge)
        net.set_params(flat(params))
        for k in (1, 2, 3, 4):
            ref, rst, rcyc, rhist, racc = cnn.solve_learned(kc, f_np, params, levels, tol=0.0, max_cycles=k, judge=judge)
            u = torch.zeros_like(f)
            st, cyc, rr, acc = homg.homg_solve_learned(s.handle, net, f, u, tol=0.0, max_cycles=k)
            assert cyc == rcyc == k
            assert acc == racc, (k, acc, racc)
            got = u.cpu().numpy()
            err = max(np.linalg.norm(got - ref) / np.linalg.norm(ref), np.abs(got - ref).max() / np.abs(ref).max())
            assert err <= LEARNED_ITERATE_TOL, (k, err)
    if c > 0:
        assert racc[0]
    else:
        assert racc == [False, False, False, False]
