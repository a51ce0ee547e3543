"""Training the learned corrector (include/homg_net.h) on error/residual pairs the solver produces.

The paper has no learned component; this module drives the library's own kernels (solver, feature,
patch-gather and training kernels) from Python, which only chooses seeds, patch corners and batch
order. For a variable-coefficient handle and a list of right-hand sides it

1. solves each problem to a tight tolerance (the reference solution u*),
2. replays the solve for c = 0, 1, 2, ... cycles to get the iterates u_c the corrector will meet,
3. forms the network input of each iterate and the scaled error (u* - u_c) / rho as the target
   (homg_features), and cuts fixed random 64 x 64 patches of both (homg_net_gather_patches),
4. trains the network with mean squared error and Adam (homg_net_train_step) over shuffled
   mini-batches of those patches.
"""

import time

import numpy as np

from . import homg


def init_params(seed, width=32, c_in=2, layers=4):
    """Seeded He-normal initial parameters in the library's flat order (per layer W[out][in][3][3],
    then b[out]); biases 0; the last layer scaled by 0.1 so an untrained network proposes small
    corrections."""
    rng = np.random.default_rng(seed)
    chans = [c_in] + [width] * (layers - 1) + [1]
    out = []
    for l in range(layers):
        co, ci = chans[l + 1], chans[l]
        w = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        if l == layers - 1:
            w *= 0.1
        out += [w.ravel(), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def make_training_set(solver, net, fs, cycles=(0, 1, 2), patches=20000, P=64, seed=0, ref_tol=1e-11):
    """Patches of network inputs and targets from the iterates of `solver` on right-hand sides `fs`
    (device FP64 tensors on the solver's grid). Returns device tensors X [N, P, 2, P, 8] (bfloat16)
    and T [N, P, P] (binary32)."""
    import torch

    n1 = fs[0].shape[0]
    rng = np.random.default_rng(seed)
    images = len(fs) * len(cycles)
    per = [patches // images + (1 if i < patches % images else 0) for i in range(images)]
    X = torch.empty(patches, P, 2, P, 8, dtype=torch.bfloat16, device="cuda")
    T = torch.empty(patches, P, P, dtype=torch.float32, device="cuda")
    x_img = torch.zeros(1, n1, 2, n1, 8, dtype=torch.bfloat16, device="cuda")
    t_img = torch.zeros(n1, n1, dtype=torch.float32, device="cuda")
    at, img = 0, 0
    for f in fs:
        ustar = torch.zeros_like(f)
        st, _, _ = solver.solve(f, ustar, tol=ref_tol, max_cycles=200)
        if st != homg.HOMG_OK:
            raise RuntimeError("reference solve did not converge")
        for c in cycles:
            u = torch.zeros_like(f)
            if c > 0:
                solver.solve(f, u, tol=0.0, max_cycles=c)
            homg.homg_features(solver.handle, f, u, x_img, u_ref=ustar, t_out=t_img)
            k = per[img]
            corners = torch.from_numpy(rng.integers(0, n1 - P + 1, size=(k, 2)).astype(np.int32)).cuda()
            net.gather_patches(x_img, t_img, corners, P, X[at:at + k], T[at:at + k])
            at += k
            img += 1
    torch.cuda.synchronize()
    return X, T


def train(net, X, T, epochs=4, batch=64, lr=1e-3, lr_final=1e-4, seed=0):
    """Adam over shuffled mini-batches; the learning rate decays geometrically from lr to lr_final.
    Returns (mean loss per epoch, seconds)."""
    import torch

    N = X.shape[0]
    rng = np.random.default_rng(seed)
    steps = epochs * (N // batch)
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    losses, step = [], 0
    Xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=X.dtype, device="cuda")
    Tb = torch.empty((batch,) + tuple(T.shape[1:]), dtype=T.dtype, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(N)).cuda()
        acc = 0.0
        for b in range(N // batch):
            idx = order[b * batch:(b + 1) * batch]
            torch.index_select(X, 0, idx, out=Xb)
            torch.index_select(T, 0, idx, out=Tb)
            acc += net.train_step(Xb, Tb, lr * decay ** step)
            step += 1
        losses.append(acc / max(1, N // batch))
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0
