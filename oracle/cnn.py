"""Learned corrector for the HOMG restart loop -- TEST INFRASTRUCTURE ONLY.

Not part of the paper, which has no learned component: a small convolutional network proposes a
correction of the current iterate from its residual before each HOMG cycle, and the plain solver
judges it (the correction is kept only when it lowers the FP64 residual norm; the HOMG cycle then
runs as usual). Plain FP64 numpy definitions, slow and direct; the GPU path shares no code with
this file. Only the test suite and the benchmark's CPU legs may import it.

Network (all 3x3 convolutions, zero padding, stride 1, channels-first arrays [C, H, W]):
    a_0 = x                                   (C_IN = 2 input channels)
    a_l = bf16(relu(conv(a_{l-1}, bf16(W_l)) + b_l))      l = 1 .. L-1   (WIDTH channels)
    y   = conv(a_{L-1}, bf16(W_L)) + b_L                   (1 channel, binary32 on the GPU)
conv(a, W)[o, i, j] = sum over c, p, q in {0, 1, 2} of W[o, c, p, q] a[c, i + p - 1, j + q - 1].
Weights are kept in binary32 ("master") and rounded to bfloat16 for every use; activations are
stored in bfloat16 after the ReLU, the way the GPU keeps them.

Input features of a node p (variable-coefficient operator, fine grid, h = 1/n):
    x_0(p) = h^2 r(p) / (D(p) rho),  x_1(p) = log k(p),
r = f - A u the FP64 residual, D(p) the sum of the four face coefficients of p (boundary nodes:
x_0 = 0), rho the root mean square of h^2 r / D over the interior nodes. The network's output y
is a correction in units of rho: u <- u + rho y at the interior nodes.

Training: mean squared error between y and the scaled true error (u* - u) / rho over a batch of
patches, gradients by the chain rule below, Adam (Kingma and Ba, 2015) on the binary32 master
weights.
"""

import numpy as np

C_IN = 2
WIDTH = 32
LAYERS = 4


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even), returned as float64: keep the top 16 bits
    of the binary32 encoding after adding 0x7fff plus the lowest kept bit."""
    a = np.atleast_1d(np.asarray(x, dtype=np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    nan = np.isnan(a)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out.reshape(np.shape(x)) if np.ndim(x) else float(out[0])


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def shapes(c_in=C_IN, width=WIDTH, layers=LAYERS):
    """(out, in) channel counts of the layers."""
    chans = [c_in] + [width] * (layers - 1) + [1]
    return [(chans[l + 1], chans[l]) for l in range(layers)]


def init_weights(seed, c_in=C_IN, width=WIDTH, layers=LAYERS):
    """He-normal weights (std sqrt(2 / (9 c_in))), zero biases, binary32 values; the last layer is
    scaled by 0.1 so an untrained network proposes small corrections."""
    rng = np.random.default_rng(seed)
    params = []
    for l, (co, ci) in enumerate(shapes(c_in, width, layers)):
        w = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        if l == layers - 1:
            w *= 0.1
        params.append((f32(w), np.zeros(co)))
    return params


def conv3x3(a, w):
    """conv(a, w)[o, i, j] = sum_{c,p,q} w[o, c, p, q] a[c, i+p-1, j+q-1], zero outside; FP64."""
    C, H, W = a.shape
    O = w.shape[0]
    pad = np.zeros((C, H + 2, W + 2))
    pad[:, 1:-1, 1:-1] = a
    y = np.zeros((O, H, W))
    for p in range(3):
        for q in range(3):
            y += np.tensordot(w[:, :, p, q], pad[:, p:p + H, q:q + W], axes=([1], [0]))
    return y


def forward(params, x, rounding=True):
    """Returns (y, activations a_0 .. a_{L-1}) for one image x [C_IN, H, W]. rounding=False skips
    every rounding (pure FP64), for derivative checks."""
    rw = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    r32 = f32 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    acts = [np.asarray(x, dtype=np.float64)]
    L = len(params)
    for l, (w, b) in enumerate(params):
        z = conv3x3(acts[-1], rw(w)) + r32(b)[:, None, None]
        if l < L - 1:
            acts.append(rw(np.maximum(z, 0.0)))
        else:
            y = r32(z[0])
    return y, acts


def patch_operator(x):
    """Weights of the Jacobi-scaled operator on one network input x [C_IN, H, W] at its inner pixels
    (not on the image border): w_q(p) = k_pq / D(p) for the four neighbours q = W, E, S, N, with k_pq
    the harmonic mean of exp(x_1) at p and q and D(p) the sum of the four. Returns [4, H-2, W-2]."""
    k = np.exp(np.asarray(x[1], dtype=np.float64))
    c = k[1:-1, 1:-1]
    faces = [face_coef(c, k[1:-1, :-2]), face_coef(c, k[1:-1, 2:]), face_coef(c, k[:-2, 1:-1]),
             face_coef(c, k[2:, 1:-1])]
    D = ((faces[0] + faces[1]) + faces[2]) + faces[3]
    return np.stack([f / D for f in faces])


def residual_loss_terms(x, y):
    """Residual of the proposal y at the inner pixels of one image, in the network's units:
    res(p) = x_0(p) - (y(p) - sum_q w_q(p) y(q)), i.e. the input's scaled residual h^2 r / (D rho)
    minus h^2 A (rho y) / (D rho), with A rebuilt from the image's own log k channel."""
    w = patch_operator(x)
    nb = [y[1:-1, :-2], y[1:-1, 2:], y[:-2, 1:-1], y[2:, 1:-1]]
    Ay = y[1:-1, 1:-1] - (((w[0] * nb[0] + w[1] * nb[1]) + w[2] * nb[2]) + w[3] * nb[3])
    return np.asarray(x[0], dtype=np.float64)[1:-1, 1:-1] - Ay, w


def loss_and_grads(params, xs, ts, rounding=True, loss_kind="error"):
    """Training loss over a batch of images and its gradient with respect to every weight and bias
    (chain rule through the ReLUs; the rounding to bfloat16 is treated as the identity, as the GPU
    does). loss_kind "error": mean squared error (1/N) sum (y - t)^2 over the N pixels against the
    scaled error t. loss_kind "residual": (1/N) sum res^2 over the N inner pixels of the images, res
    the residual left by the proposal (residual_loss_terms); t is not used."""
    L = len(params)
    if loss_kind == "error":
        npix = sum(t.size for t in ts)
    else:
        npix = sum((x.shape[1] - 2) * (x.shape[2] - 2) for x in xs)
    gw = [np.zeros_like(w) for w, _ in params]
    gb = [np.zeros_like(b) for _, b in params]
    loss = 0.0
    for x, t in zip(xs, ts):
        y, acts = forward(params, x, rounding)
        if loss_kind == "error":
            dy = y - t
            loss += float(np.sum(dy * dy))
            g = (2.0 / npix) * dy[None]  # d loss / d z_L
        else:
            res, w = residual_loss_terms(x, y)
            loss += float(np.sum(res * res))
            # d res(p) / d y(p) = -1, d res(p) / d y(q) = w_q(p) for the neighbours q of p
            gy = np.zeros_like(y)
            gy[1:-1, 1:-1] -= res
            gy[1:-1, :-2] += w[0] * res
            gy[1:-1, 2:] += w[1] * res
            gy[:-2, 1:-1] += w[2] * res
            gy[2:, 1:-1] += w[3] * res
            g = (2.0 / npix) * gy[None]
        for l in range(L - 1, -1, -1):
            a = acts[l]
            C, H, W = a.shape
            pad = np.zeros((C, H + 2, W + 2))
            pad[:, 1:-1, 1:-1] = a
            for p in range(3):
                for q in range(3):
                    gw[l][:, :, p, q] += np.tensordot(g, pad[:, p:p + H, q:q + W], axes=([1, 2], [1, 2]))
            gb[l] += g.sum(axis=(1, 2))
            if l > 0:
                # d loss / d a_{l-1} = conv with the kernel flipped in space and transposed in channels
                wl = bf16(params[l][0]) if rounding else params[l][0]
                wt = wl[:, :, ::-1, ::-1].transpose(1, 0, 2, 3)
                da = conv3x3(g, wt)
                g = da * (a > 0)
    return loss / npix, gw, gb


def adam(params, grads_w, grads_b, state, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step = 1, 2, ...): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    w <- w - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); weights kept in binary32."""
    if state is None:
        state = [[np.zeros_like(w), np.zeros_like(w), np.zeros_like(b), np.zeros_like(b)] for w, b in params]
    out = []
    for (w, b), gw, gb, st in zip(params, grads_w, grads_b, state):
        new = []
        for val, g, mi in ((w, gw, 0), (b, gb, 2)):
            st[mi] = beta1 * st[mi] + (1 - beta1) * g
            st[mi + 1] = beta2 * st[mi + 1] + (1 - beta2) * g * g
            mhat = st[mi] / (1 - beta1 ** step)
            vhat = st[mi + 1] / (1 - beta2 ** step)
            new.append(f32(val - lr * mhat / (np.sqrt(vhat) + eps)))
        out.append((new[0], new[1]))
    return out, state


def face_coef(a, b):
    return (2.0 * a) * b / (a + b)


def diagonal(kc):
    """D(p) = ((k_W + k_E) + k_S) + k_N at the interior nodes (0 on the boundary)."""
    D = np.zeros_like(kc)
    c = kc[1:-1, 1:-1]
    kw = face_coef(c, kc[1:-1, :-2])
    ke = face_coef(c, kc[1:-1, 2:])
    ks = face_coef(c, kc[:-2, 1:-1])
    kn = face_coef(c, kc[2:, 1:-1])
    D[1:-1, 1:-1] = ((kw + ke) + ks) + kn
    return D


def features(kc, r):
    """Network input [2, n+1, n+1] (bfloat16 values) and the scale rho from the FP64 residual r."""
    n = kc.shape[0] - 1
    h2 = (1.0 / n) ** 2
    D = diagonal(kc)
    z = np.zeros_like(r)
    z[1:-1, 1:-1] = h2 * r[1:-1, 1:-1] / D[1:-1, 1:-1]
    rho = np.sqrt(np.mean(z[1:-1, 1:-1] ** 2))
    x = np.zeros((2,) + r.shape)
    x[0] = bf16(z / rho) if rho > 0 else 0.0
    x[1] = bf16(np.log(kc))
    return x, rho


def solve_learned(kc, f, params, levels, precision="fp64", tol=1e-10, max_cycles=100, div_factor=1e3,
                  judge="proposal"):
    """Restarted variable-coefficient HOMG solve with the learned corrector ahead of every cycle:
    r = f - A u; if ||r|| / ||f|| <= tol stop; propose u' = u + rho y (interior) from the network;
    judge (the plain solver decides, in FP64 residual norms):
      judge "proposal":    keep u' when ||f - A u'|| < ||r||, then one HOMG cycle on the residual
                           of the kept iterate;
      judge "after_cycle": run one HOMG cycle from u and one from u', keep the result with the
                           smaller residual norm.
    After two rejections in a row the network proposes nothing more (plain cycles only).
    Returns (u, status, cycles, hist, accepted) with accepted[k] the judge's decision at cycle k
    (False for a cycle without a proposal)."""
    from . import oracle as o

    u = np.zeros_like(f)
    fnorm = o.norm_interior(f)
    if fnorm == 0.0:
        return u, o.OK, 0, np.zeros(1), []
    hist, accepted = [], []
    rr0 = None
    k = 0
    rejected_in_a_row = 0

    def after_cycle(v, rv):
        w = v.copy()
        e = o.cycle_vc(kc, rv, levels, precision=precision)
        w[1:-1, 1:-1] += e[1:-1, 1:-1]
        return w

    while True:
        r = o.residual_vc(kc, f, u)
        rn = o.norm_interior(r)
        rr = rn / fnorm
        hist.append(rr)
        rr0 = rr if rr0 is None else rr0
        if rr <= tol:
            return u, o.OK, k, np.array(hist), accepted
        if not np.isfinite(rr) or rr > div_factor * rr0:
            return u, o.DIVERGED, k, np.array(hist), accepted
        if k == max_cycles:
            return u, o.NOT_CONVERGED, k, np.array(hist), accepted
        if rejected_in_a_row >= 2:
            accepted.append(False)
            u = after_cycle(u, r)
            k += 1
            continue
        x, rho = features(kc, r)
        y, _ = forward(params, x)
        u2 = u.copy()
        u2[1:-1, 1:-1] += rho * y[1:-1, 1:-1]
        r2 = o.residual_vc(kc, f, u2)
        if judge == "proposal":
            keep = o.norm_interior(r2) < rn
            if keep:
                u, r = u2, r2
            u = after_cycle(u, r)
        else:
            up = after_cycle(u, r)
            uq = after_cycle(u2, r2)
            keep = o.norm_interior(o.residual_vc(kc, f, uq)) < o.norm_interior(o.residual_vc(kc, f, up))
            u = uq if keep else up
        accepted.append(bool(keep))
        rejected_in_a_row = 0 if keep else rejected_in_a_row + 1
        k += 1
