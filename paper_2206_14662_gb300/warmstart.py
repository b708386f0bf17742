"""Training and evaluation of the learned field-solve warm start.

Snapshots come from the method itself: a batch of simulations with
randomised pressure, voltage and field is stepped, and after every step the
pair (this step's node charge, the previous space-charge potential) ->
(the change of the space-charge potential) is kept on the device.  The net
(libpic's pic_unet_*) is trained on them with its own forward and backward
kernels; used in the loop (warm_start = 2) it supplies the initial guess
phi_prev + dphi_scale * net(rho / rho_scale, phi_prev / phi_scale), which the
field solve refines to the same residual bound as without it.

Tensors here are torch CUDA tensors used as device buffers; the network's
arithmetic runs in the library.
"""
from __future__ import annotations

import numpy as np

from .inputs import seed_particles, workload


def snapshot_configs(n_sims: int, nr: int = 128, nz: int = 512, n_particles: int = 10_000,
                     seed: int = 0, **over) -> list[dict]:
    """The small workload's physics (coax, uniform B_z) on an nr x nz grid,
    with pressure log-uniform in [1e-5, 1e-3] mbar, inner voltage uniform in
    [-20, -5] kV and B0 uniform in [0.1, 0.5] T per simulation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cfgs = []
    for _ in range(n_sims):
        c = workload("coax_32x64_1e4", nr=nr, nz=nz, n_init=n_particles, precision=32,
                     p_mbar=float(10 ** rng.uniform(-5, -3)),
                     v_inner=float(rng.uniform(-20e3, -5e3)),
                     b0=float(rng.uniform(0.1, 0.5)), sort_every=20)
        c.update(over)
        cfgs.append(c)
    return cfgs


def collect(cfgs: list[dict], steps: int, warmup: int = 0, seed: int = 0):
    """Step the batch and keep (rho, phi_prev, dphi) of every simulation and
    step: three float32 CUDA tensors (n, nr, nz), n = len(cfgs) * steps."""
    import torch
    from ._capi import Simulation
    S, nr, nz = len(cfgs), cfgs[0]["nr"], cfgs[0]["nz"]
    rho = torch.empty((steps, S, nr, nz), dtype=torch.float32, device="cuda")
    prev = torch.empty_like(rho)
    new = torch.empty_like(rho)
    with Simulation(cfgs) as sim:
        for k, c in enumerate(cfgs):
            sim.load_particles(*seed_particles(c, seed=seed * 1000 + k), sim=k)
        sim.step(warmup)
        for s in range(steps):
            sim.field_images(None, prev[s])
            sim.step(1)
            sim.field_images(rho[s], new[s])
    n = steps * S
    return rho.reshape(n, nr, nz), prev.reshape(n, nr, nz), (new - prev).reshape(n, nr, nz)


def scales(rho, phi, dphi) -> tuple[float, float, float]:
    """RMS of each quantity over the data set."""
    f = lambda t: float(t.double().pow(2).mean().sqrt().item()) or 1.0
    return f(rho), f(phi), f(dphi)


def train(net, rho, phi, dphi, sc, epochs: int = 1, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam over shuffled mini-batches of the net's batch size; returns the
    loss of each step and the loss a zero prediction (no change of the
    potential) would have on the same batch (float32 CUDA tensors)."""
    import torch
    B = net.shape[0]
    n = rho.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.empty(net.shape + (2,), dtype=torch.float32, device="cuda")
    t = torch.empty(net.shape, dtype=torch.float32, device="cuda")
    steps = epochs * (n // B)
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    base = torch.zeros(steps, dtype=torch.float32, device="cuda")
    k = 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        for i in range(n // B):
            idx = perm[i * B:(i + 1) * B]
            x[..., 0] = rho[idx] / sc[0]
            x[..., 1] = phi[idx] / sc[1]
            t.copy_(dphi[idx] / sc[2])
            net.train_step(x, t, lr=lr, loss=losses[k:k + 1])
            base[k] = 0.5 * t.pow(2).mean()
            k += 1
            if log_every and k % log_every == 0:
                print(f"step {k} loss {losses[k - 1].item():.4e}", flush=True)
    return losses, base


def evaluate(cfg: dict, steps: int, net=None, sc=None, seed: int = 0, warmup: int = 0):
    """One simulation stepped with the previous potential as the initial
    guess (net None) or with the net: per step the initial guess' relative
    residual, the sweeps and the final residual."""
    from ._capi import Simulation
    c = dict(cfg, warm_start=2 if net is not None else 1)
    out = {"relres_init": [], "sweeps": [], "relres": []}
    with Simulation(c) as sim:
        sim.load_particles(*seed_particles(c, seed=seed))
        sim.step(warmup)
        if net is not None:
            sim.attach_unet(net, *sc)
        for _ in range(steps):
            sim.step(1)
            d = sim.diagnostics()
            out["relres_init"].append(d["poisson_relres_init"])
            out["sweeps"].append(d["poisson_iters"])
            out["relres"].append(d["poisson_relres"])
        if net is not None:
            sim.attach_unet(None, 1.0, 1.0, 1.0)
    return {k: np.array(v) for k, v in out.items()}


def forward_flops(c: int, H: int, W: int) -> float:
    """Multiply-adds x 2 of one forward pass on an H x W image (real
    channel counts): 3 x 3 layers 18 in out pixels, transposed layers
    8 in out coarse pixels, the head 2 c pixels."""
    P = [H * W, H * W // 4, H * W // 16, H * W // 64]
    w = [c, 2 * c, 4 * c, 8 * c]
    f = 18.0 * P[0] * (2 * c + c * c)                     # level 1 encoder
    for k in (1, 2, 3):
        f += 18.0 * P[k] * (w[k - 1] * w[k] + w[k] * w[k])   # levels 2..4 encoder
    for k in (2, 1, 0):                                   # decoder levels 3, 2, 1
        f += 8.0 * P[k + 1] * w[k + 1] * w[k]             # transposed 2 x 2
        f += 18.0 * P[k] * (2 * w[k] * w[k] + w[k] * w[k])
    f += 2.0 * P[0] * c
    return f


def train_step_flops(c: int, H: int, W: int, batch: int) -> float:
    """Forward, data gradients and weight gradients: three times the forward
    (the first layer's data gradient is not formed; ignored)."""
    return 3.0 * batch * forward_flops(c, H, W)
