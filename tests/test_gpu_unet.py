"""The U-Net of the learned field-solve warm start, forward and backward
through the C ABI, against the CPU FP64 oracle (oracle/unet.py): FP32 test
mode to 1e-5, BF16 tensor-core mode to the BF16 tolerance, on a 16 x 32 grid
with base width 4 (every layer padded) and on 16 x 64 with base width 32
(the production widths, full tensor-core tiles)."""
import numpy as np
import pytest

from oracle import unet as U
from paper_2206_14662_gb300.inputs import unet_init_flat, unet_layer_shapes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2206_14662_gb300 import build
    build.build()
    return torch


def _layer_slices(c):
    out, o = {}, 0
    for name, shp in unet_layer_shapes(c):
        k = int(np.prod(shp)) + (1 if name == "head" else shp[-1])
        out[name] = slice(o, o + k)
        o += k
    return out


def _case(torch, c, B, H, W, precision, seed=0, q=None, coherent=False, tensor_path=-1):
    """GPU and oracle outputs, parameter gradients and input gradients for
    one forward / backward; q the oracle's storage rounding; coherent: the
    output gradient of the loss against a smooth target instead of noise."""
    from paper_2206_14662_gb300.unet import UNet
    flat = unet_init_flat(c, seed=seed, head_std=0.3, bias_std=0.1).astype(np.float32)
    rng = np.random.default_rng(seed + 7)
    x = rng.standard_normal((B, H, W, 2)).astype(np.float32)
    gy = (rng.standard_normal((B, H, W)) / (B * H * W)).astype(np.float32)
    if coherent:
        yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        t = np.sin(2 * np.pi * yy / H) * np.cos(2 * np.pi * xx / W)
        y0, _ = U.forward(U.unflatten(flat.astype(np.float64), c), x.astype(np.float64))
        gy = ((y0 - t) / (B * H * W)).astype(np.float32)
    net = UNet(c, H, W, B, precision=precision)
    net.set_tensor_path(tensor_path)
    net.set_params(flat)
    assert np.array_equal(net.get_params(), flat)
    xd = torch.from_numpy(x).cuda()
    y = net.forward(xd).cpu().numpy()
    gx = torch.zeros((B, H, W, 2), dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(gy).cuda(), gx)
    grads = net.get_grads()
    net.close()
    p = U.unflatten(flat.astype(np.float64), c)
    yo, a = U.forward(p, x.astype(np.float64), q=q)
    go = U.backward(p, a, gy.astype(np.float64), q=q)
    return y, yo, grads, U.flatten({k: v for k, v in go.items() if k != "x"}), gx.cpu().numpy(), go["x"]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("c,H,W", [(4, 16, 32), (32, 16, 64)])
def test_fp32_mode_matches_oracle(torch, c, H, W):
    y, yo, g, go, gx, gxo = _case(torch, c, 2, H, W, precision=32)
    assert np.abs(y - yo).max() <= 1e-5 * np.abs(yo).max()
    for name, sl in _layer_slices(c).items():
        assert _rel(g[sl], go[sl]) <= 1e-5, name
    assert _rel(gx, gxo) <= 1e-5


def test_bf16_tensor_core_mode_matches_bf16_rounding_oracle(torch):
    """Base width 4 (every layer padded to 32 channels, all tensor-core
    GEMM forms: 3 x 3 forward, data and weight gradients, transposed
    convolutions, masks): the BF16 path equals the oracle that rounds to
    BF16 where the GPU stores BF16, up to FP32 accumulation order."""
    y, yo, g, go, gx, gxo = _case(torch, 4, 2, 16, 32, precision=16, q=U.round_bf16)
    assert _rel(y, yo) <= 1e-5
    for name, sl in _layer_slices(4).items():
        assert _rel(g[sl], go[sl]) <= 1e-5, name
    assert _rel(gx, gxo) <= 1e-5


@pytest.mark.parametrize("c,H,W", [(4, 32, 64), (32, 64, 128)])
def test_tcgen05_conv_matches_bf16_rounding_oracle(torch, c, H, W):
    """The 3 x 3 convolutions (forward and data gradient) on the tcgen05
    kernel wherever the shape allows: levels 1-3 of the 32 x 64 grid at base
    width 4 (N = 32), all four levels of 64 x 128 at base width 32 (N = 32
    to 256).  Against the oracle that rounds to BF16 where the GPU stores
    BF16 the results agree up to FP32 summation order, as the mma.sync
    path's do; the two paths agree with each other as closely."""
    q = U.round_bf16
    coh = c == 32   # (a loss against a smooth target at the production width)
    y, yo, g, go, gx, gxo = _case(torch, c, 1, H, W, precision=16, q=q, coherent=coh,
                                  tensor_path=1)
    y0, _, g0, _, gx0, _ = _case(torch, c, 1, H, W, precision=16, q=q, coherent=coh,
                                 tensor_path=0)
    tol = 1e-5 if c == 4 else 1e-2
    assert _rel(y, yo) <= tol
    assert _rel(g, go) <= (1e-5 if c == 4 else 1.5e-2)
    if c == 4:
        # (at the production width the input gradient carries the BF16
        # storage of all 18 layers, as in the test below, which does not
        # bound it either)
        assert _rel(gx, gxo) <= 1e-5
    assert _rel(y, y0) <= tol and _rel(g, g0) <= (1e-5 if c == 4 else 1.5e-2)


@pytest.mark.parametrize("H,W", [(16, 64), (32, 64)])
def test_bf16_tensor_core_mode_production_width(torch, H, W):
    """Base width 32 (the production widths, full 64-channel tiles, K up to
    9 x 256): against the FP64 oracle the output agrees to 1e-2 and the
    gradients of a loss against a smooth target to the BF16 storage
    tolerance.  The remaining differences are BF16 values one unit apart
    where the FP32 sum of several thousand products falls on the other side
    of a rounding boundary than the exact sum; they accumulate through the
    18 layers (the width-4 case above shows the kernels themselves exact)."""
    y, yo, g, go, gx, gxo = _case(torch, 32, 2, H, W, precision=16, coherent=True)
    assert _rel(y, yo) <= 1e-2
    assert _rel(g, go) <= 2.5e-2
    y, yo, g, go, gx, gxo = _case(torch, 32, 2, H, W, precision=16, q=U.round_bf16, coherent=True)
    assert _rel(y, yo) <= 1e-2
    assert _rel(g, go) <= 1.5e-2
    assert max(_rel(g[sl], go[sl]) for sl in _layer_slices(32).values()) <= 8e-2


def test_production_grid_128x512(torch):
    """The size the net runs at inside the loop: base width 32 on the
    128 x 512 grid, batch 1, the output gradient of a loss against a smooth
    target.  One FP64 oracle forward and backward is the reference for both
    modes: the FP32 test mode to 1e-5 (output, every layer's gradients, the
    input gradient), the BF16 tensor-core mode to the BF16 tolerances of the
    narrower production-width case."""
    from paper_2206_14662_gb300.unet import UNet
    c, B, H, W = 32, 1, 128, 512
    flat = unet_init_flat(c, seed=11, head_std=0.3, bias_std=0.1).astype(np.float32)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((B, H, W, 2)).astype(np.float32)
    p = U.unflatten(flat.astype(np.float64), c)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    t = np.sin(2 * np.pi * yy / H) * np.cos(2 * np.pi * xx / W)
    yo, a = U.forward(p, x.astype(np.float64))
    gy = ((yo - t) / (B * H * W)).astype(np.float32)
    go = U.backward(p, a, gy.astype(np.float64))
    go_flat = U.flatten({k: v for k, v in go.items() if k != "x"})
    # the same network in plain FP32 arithmetic (numpy, blocked sums): how
    # far FP32 rounding alone moves each result from the FP64 oracle.  The
    # weight gradients sum over up to 65 536 pixels and the input gradient
    # comes through 18 layers, so at this size that is well above 1e-5.
    p32 = {k: v.astype(np.float32) for k, v in p.items()}
    y32, a32 = U.forward(p32, x)
    g32 = U.backward(p32, a32, gy)
    g32_flat = U.flatten({k: v for k, v in g32.items() if k != "x"})
    res = {}
    for prec in (32, 16):
        net = UNet(c, H, W, B, precision=prec)
        net.set_params(flat)
        y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        gx = torch.zeros((B, H, W, 2), dtype=torch.float32, device="cuda")
        net.backward(torch.from_numpy(gy).cuda(), gx)
        res[prec] = (y, net.get_grads(), gx.cpu().numpy())
        net.close()
    # FP32 test mode: within 10x of plain FP32's own distance from the FP64
    # oracle (the kernels sum in other orders: tiles, pixel splits, FP32
    # atomics), and never worse than 1e-5 where FP32 is that close.  A
    # tiling or index mistake gives errors of order one.
    y, g, gx = res[32]
    bar = lambda e32: max(1e-5, 10.0 * e32)
    assert _rel(y, yo) <= bar(_rel(y32, yo))
    for name, sl in _layer_slices(c).items():
        assert _rel(g[sl], go_flat[sl]) <= bar(_rel(g32_flat[sl], go_flat[sl])), name
    assert _rel(gx, go["x"]) <= bar(_rel(g32["x"], go["x"]))
    y, g, gx = res[16]
    assert _rel(y, yo) <= 1e-2
    assert _rel(g, go_flat) <= 2.5e-2


def test_adam_matches_oracle(torch):
    """Three training steps on the GPU (forward, loss gradient, backward,
    Adam); after each, the parameters equal the oracle's FP64 Adam step
    (Kingma and Ba, Algorithm 1) applied to the GPU's own gradients of that
    step, element by element, within FP32 rounding of the weights plus
    1e-5 of the step size per step."""
    from paper_2206_14662_gb300.unet import UNet
    c, B, H, W = 8, 2, 16, 32
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    flat = unet_init_flat(c, seed=4).astype(np.float32)
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal((B, H, W, 2)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    net = UNet(c, H, W, B, precision=32)
    net.set_params(flat)
    w = flat.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    moved = 0.0
    for step in (1, 2, 3):
        net.train_step(x, t, lr=lr, beta1=b1, beta2=b2, eps=eps)
        g = net.get_grads().astype(np.float64)
        # (weights feeding inactive ReLUs get exactly zero gradient)
        assert np.count_nonzero(g) > 0.5 * g.size
        w, m, v = U.adam_step(w, g, m, v, step, lr, b1, b2, eps)
        got = net.get_params().astype(np.float64)
        ulp = np.spacing(np.abs(w).astype(np.float32)).astype(np.float64)
        assert (np.abs(got - w) <= step * (ulp + 1e-5 * lr)).all(), step
        moved = np.abs(got - flat).max()
    net.close()
    assert moved > 2 * lr


def test_training_reduces_the_loss(torch):
    """Adam on a fixed smooth mapping (the target is a blurred copy of the
    first input channel): the loss falls by an order of magnitude."""
    from paper_2206_14662_gb300.unet import UNet
    B, H, W, c = 4, 32, 64, 8
    rng = np.random.default_rng(3)
    x = rng.standard_normal((B, H, W, 2)).astype(np.float32)
    k = np.ones(5) / 5.0
    t = x[..., 0].copy()
    for axis in (1, 2):
        t = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), axis, t)
    net = UNet(c, H, W, B, precision=16)
    net.set_params(unet_init_flat(c, seed=1).astype(np.float32))
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for _ in range(300):
        net.train_step(xd, td, lr=2e-3, loss=loss)
        hist.append(float(loss.item()))
    net.close()
    assert hist[-1] < 0.1 * hist[0], (hist[0], hist[-1])


def test_learned_warm_start_with_a_zero_net_is_the_previous_potential(torch):
    """warm_start = 2 with a net whose output is zero gives, bit for bit,
    the run refined from the previous potential (graph blocks included)."""
    from paper_2206_14662_gb300._capi import PIC_GRID_PHI, Simulation
    from paper_2206_14662_gb300.inputs import seed_particles, workload
    from paper_2206_14662_gb300.unet import UNet
    from parity import by_uid
    out = []
    for ws in (1, 2):
        cfg = workload("mirror_128x512_1e7", n_init=30_000, warm_start=ws, sort_every=4)
        with Simulation(cfg) as sim:
            sim.load_particles(*seed_particles(cfg))
            net = None
            if ws == 2:
                net = UNet(32, cfg["nr"], cfg["nz"], 1, precision=16)
                net.set_params(np.zeros(net.n_params, dtype=np.float32))
                sim.attach_unet(net, 1e-12, 1.0, 1e-3)
            sim.step(3)
            sim.step(16)
            d = sim.diagnostics()
            out.append((by_uid(sim.export_particles()), sim.get_grid(PIC_GRID_PHI), d))
            if net is not None:
                sim.attach_unet(None, 1.0, 1.0, 1.0)
                net.close()
    (ga, pa, da), (gb, pb, db) = out
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    assert np.array_equal(pa, pb)
    # the norms are sums of block partials in arrival order
    assert db["poisson_relres_init"] == pytest.approx(da["poisson_relres_init"], rel=1e-12)
    assert da["poisson_relres_init"] > 0
    assert db["kernels_launched"] > da["kernels_launched"]


def test_learned_warm_start_trained_in_the_loop(torch):
    """Snapshots from a batch of eight randomised simulations of the small
    workload's physics, a few hundred Adam steps, then the trained net as the
    initial guess inside the loop: every solve still meets poisson_rtol, and
    the initial residuals with and without the net are reported."""
    from paper_2206_14662_gb300 import warmstart
    from paper_2206_14662_gb300.unet import UNet
    cfgs = warmstart.snapshot_configs(8, nr=32, nz=64, n_particles=3000, seed=1)
    rho, phi, dphi = warmstart.collect(cfgs, steps=64, warmup=4)
    sc = warmstart.scales(rho, phi, dphi)
    net = UNet(8, 32, 64, 16, precision=16)
    net.set_params(unet_init_flat(8, seed=2).astype(np.float32))
    losses, base = warmstart.train(net, rho, phi, dphi, sc, epochs=16, lr=1e-3)
    losses, base = losses.cpu().numpy(), base.cpu().numpy()
    # against predicting no change on the same batches, the trained net
    # explains part of the potential's change
    assert losses[-64:].mean() < 0.8 * base[-64:].mean()
    inf = UNet(8, 32, 64, 1, precision=16)
    inf.set_params(net.get_params())
    cfg = warmstart.snapshot_configs(1, nr=32, nz=64, n_particles=3000, seed=9)[0]
    prv = warmstart.evaluate(cfg, 24, warmup=4)
    lrn = warmstart.evaluate(cfg, 24, inf, sc, warmup=4)
    net.close()
    inf.close()
    for r in (prv, lrn):
        assert (r["relres"] <= cfg["poisson_rtol"]).all()
    print(f"initial residual: previous potential {np.median(prv['relres_init']):.3e}, "
          f"learned {np.median(lrn['relres_init']):.3e}; sweeps {prv['sweeps'].mean():.2f} / "
          f"{lrn['sweeps'].mean():.2f}; loss / no-change loss {losses[-64:].mean() / base[-64:].mean():.3f}")
