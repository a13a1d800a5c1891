"""Learned warm start for Algorithm 3 (an addition to the paper's method).

A U-Net (`wdb.WarmStartNet`, kernels in csrc/cnn.cu) is trained to map an observation u0 to
the image Psi x* of the minimiser x* of the l1-l2 problem for one blur (one Theta_K). At
solve time `WarmStartNet.solve_warm` starts FISTA from Psi* network(u0) when that start has a
lower objective than x = 0 (else it falls back to x = 0), and the caller's stopping rule is
unchanged, so the returned x solves the same problem; only the number of iterations changes.

This module is the host driver: it draws observations from the seeded generator, computes
x* with the library's own solver, and runs the training loop. Every arithmetic step (solver,
transforms, forward, backward, Adam) runs in libwdb's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synthetic
from . import wdb


def observations(n: int, psf: np.ndarray, count: int, config_id: int, first: int = 0, noise: float = 0.01):
    """`count` seeded observations u0 = H u + b (instances first .. first+count-1)."""
    return [synthetic.make_problem(n, psf, 0.0, config_id, first + i, noise=noise).u0 for i in range(count)]


def _observation_job(args):
    n, psf, config_id, instance, noise = args
    return synthetic.make_problem(n, psf, 0.0, config_id, instance, noise=noise).u0.astype(np.float32)


def observations_mixed(n: int, psfs, per_blur: int, config_id: int, noise: float = 0.01, workers: int = 1):
    """per_blur seeded observations for each blur, blur-major (instance = blur index * per_blur
    + image index), as a float32 array [len(psfs) * per_blur, n, n]; workers > 1 spreads the
    synthesis over spawned processes."""
    jobs = [(n, psf, config_id, k * per_blur + i, noise) for k, psf in enumerate(psfs) for i in range(per_blur)]
    if workers <= 1:
        return np.stack([_observation_job(j) for j in jobs])
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
        return np.stack(list(pool.map(_observation_job, jobs, chunksize=64)))


def solution_images_batched(thetas, U, lam: float, iters: int, tol: float = 0.0, precond: str = "spai",
                            wavelet: str = "db4"):
    """Targets Psi x* for observations U [len(thetas) * per_blur, n, n] (blur-major, problem
    k * per_blur + i uses thetas[k]): x* from the batched solver (one problem per blur handle
    per call, `iters` iterations or the relative gap `tol`), then one IDWT each."""
    import torch
    nb = len(thetas)
    M = U.shape[0]
    per = M // nb
    n_rows, n_cols, J = thetas[0].info.n_rows, thetas[0].info.n_cols, thetas[0].info.levels
    N = n_rows * n_cols
    X = torch.zeros(nb, N, device="cuda")
    T = torch.empty(M, n_rows, n_cols, device="cuda")
    Uf = U.view(M, N)
    params = [dict(lam=lam, max_iters=iters, tol=tol, precond=precond, check_every=20)] * nb
    iters_run = []
    for i in range(per):
        X.zero_()
        res = wdb.solve_batch(thetas, [Uf[k * per + i] for k in range(nb)], [X[k] for k in range(nb)], params)
        iters_run += [r["iters"] for r in res]
        for k in range(nb):
            wdb.idwt(X[k], T[k * per + i].view(-1), n_rows, n_cols, wavelet, J)
    return T, iters_run


def _stack(arrs):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.stack(arrs), dtype=np.float32)).cuda()


def solution_images(theta: wdb.Theta, u0s, lam: float, iters: int, precond: str = "spai", levels: int | None = None,
                    wavelet: str = "db4"):
    """Targets Psi x* for each observation: x* from `iters` FISTA iterations on Theta_K."""
    import torch
    n_rows, n_cols = theta.info.n_rows, theta.info.n_cols
    J = theta.info.levels if levels is None else levels
    out = []
    x = torch.zeros(theta.N, device="cuda")
    img = torch.zeros(theta.N, device="cuda")
    for u0 in u0s:
        u = _stack([u0]).view(-1)
        theta.solve(u, x, lam=lam, max_iters=iters, precond=precond)
        wdb.idwt(x, img, n_rows, n_cols, wavelet, J)
        out.append(img.view(n_rows, n_cols).clone())
    return torch.stack(out)


@dataclass
class TrainLog:
    losses: list
    seconds: float


def train(net: wdb.WarmStartNet, U, T, steps: int, batch: int, lr: float = 1e-3, seed: int = 0,
          decay_at: float = 0.75) -> TrainLog:
    """Adam on mean squared error over random mini-batches of (U, T) ([M, H, W] CUDA tensors).
    The learning rate drops 10x after `decay_at` of the steps."""
    import time
    import torch
    rng = np.random.default_rng(seed)
    M = U.shape[0]
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        idx = torch.from_numpy(rng.choice(M, size=min(batch, M), replace=False)).cuda()
        u = U.index_select(0, idx).contiguous()
        t = T.index_select(0, idx).contiguous()
        losses.append(net.train_step(u, t, lr if s < decay_at * steps else 0.1 * lr))
    torch.cuda.synchronize()
    return TrainLog(losses, time.perf_counter() - t0)


def reference_objective(theta: wdb.Theta, u, lam: float, iters: int = 3000, precond: str = "spai") -> float:
    """E* estimate: the objective after a long solve."""
    import torch
    x = torch.zeros(theta.N, device="cuda")
    return theta.solve(u, x, lam=lam, max_iters=iters, precond=precond)["objective"]


def iterations_to_target(theta, net, u, lam, E_star, rel, precond="spai", max_iters=5000):
    """Iterations to reach E <= E*(1 + rel) from x = 0, from Psi* u and from the network's
    start (solve_warm). Returns a dict of the three counts and the start solve_warm chose."""
    import torch
    target = E_star * (1.0 + rel)
    x = torch.zeros(theta.N, device="cuda")
    kw = dict(lam=lam, max_iters=max_iters, precond=precond, target_objective=target)
    cold = theta.solve(u, x, **kw)
    x0 = torch.zeros(theta.N, device="cuda")
    J, nr, nc = theta.info.levels, theta.info.n_rows, theta.info.n_cols
    wdb.dwt(u, x0, nr, nc, "db4", J)
    obs = theta.solve(u, x, x_init=x0, **kw)
    r, used = net.solve_warm(theta, u, x, **kw)
    return {"cold": cold["first_primal_below"] or cold["iters"], "obs": obs["first_primal_below"] or obs["iters"],
            "warm": r["first_primal_below"] or r["iters"], "start": used, "warm_objective": r["objective"]}
