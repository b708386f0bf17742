"""CPU FP64 oracle of the learned initial guess for the field solve: a
four-level convolutional U-Net and its gradients, written out with numpy.

TEST INFRASTRUCTURE ONLY: tests/ and bench.py's cpu legs may use this
module; the product path never does.  It shares no code with the CUDA
library.  The paper has no counterpart: the network is this library's
optional warm start of the field solve, which still iterates to the same
residual bound.

Network (base width c, input channels cin, H and W divisible by 8):
  level 1 (H x W):        e1a = relu(conv3(x,   2 -> c)),  s1 = relu(conv3(e1a, c -> c))
  level 2 (H/2 x W/2):    e2a = relu(conv3(pool(s1), c -> 2c)), s2 = relu(conv3(e2a))
  level 3 (H/4 x W/4):    e3a = relu(conv3(pool(s2), 2c -> 4c)), s3 = relu(conv3(e3a))
  level 4 (H/8 x W/8):    e4a = relu(conv3(pool(s3), 4c -> 8c)), e4b = relu(conv3(e4a))
  decoder, k = 3, 2, 1:   u_k = upconv2(previous, -> width of level k)
                          d_ka = relu(conv3(concat(u_k, s_k))), d_kb = relu(conv3(d_ka))
  head:                   y = d1b . w_head + b_head   (1 x 1 convolution to one channel)
conv3 is a 3 x 3 cross-correlation with zero padding and bias,
out[y, x] = b + sum_{ky, kx} in[y + ky - 1, x + kx - 1] W[ky, kx]; pool the
mean over 2 x 2 blocks; upconv2 the transposed 2 x 2 convolution of stride
2, out[2y + dy, 2x + dx] = in[y, x] U[dy, dx] + b; concat puts the upsampled
channels first.  Arrays are (batch, H, W, channels).  The loss is
L = sum (y - t)^2 / (2 N), N the number of output values.
"""
from __future__ import annotations

import numpy as np

CONV_LAYERS = ("enc1a", "enc1b", "enc2a", "enc2b", "enc3a", "enc3b", "enc4a", "enc4b",
               "dec3a", "dec3b", "dec2a", "dec2b", "dec1a", "dec1b")
UP_LAYERS = ("up3", "up2", "up1")
# parameter order of the flat vector (weights, then bias, per layer)
LAYER_ORDER = ("enc1a", "enc1b", "enc2a", "enc2b", "enc3a", "enc3b", "enc4a", "enc4b",
               "up3", "dec3a", "dec3b", "up2", "dec2a", "dec2b", "up1", "dec1a", "dec1b",
               "head")


def layer_shapes(c: int, cin: int = 2) -> dict:
    """Weight shape of every layer: conv (3, 3, in, out), upconv
    (2, 2, in, out), head (c,)."""
    s = {"enc1a": (3, 3, cin, c), "enc1b": (3, 3, c, c),
         "enc2a": (3, 3, c, 2 * c), "enc2b": (3, 3, 2 * c, 2 * c),
         "enc3a": (3, 3, 2 * c, 4 * c), "enc3b": (3, 3, 4 * c, 4 * c),
         "enc4a": (3, 3, 4 * c, 8 * c), "enc4b": (3, 3, 8 * c, 8 * c),
         "up3": (2, 2, 8 * c, 4 * c), "dec3a": (3, 3, 8 * c, 4 * c), "dec3b": (3, 3, 4 * c, 4 * c),
         "up2": (2, 2, 4 * c, 2 * c), "dec2a": (3, 3, 4 * c, 2 * c), "dec2b": (3, 3, 2 * c, 2 * c),
         "up1": (2, 2, 2 * c, c), "dec1a": (3, 3, 2 * c, c), "dec1b": (3, 3, c, c),
         "head": (c,)}
    return s


def flatten(params: dict) -> np.ndarray:
    """Parameters in the flat order: per layer of LAYER_ORDER its weights
    (C order) then its bias."""
    return np.concatenate([np.concatenate([params[n + ".w"].ravel(), np.atleast_1d(params[n + ".b"]).ravel()])
                           for n in LAYER_ORDER])


def unflatten(vec: np.ndarray, c: int, cin: int = 2) -> dict:
    out, o = {}, 0
    for n, shp in layer_shapes(c, cin).items():
        k = int(np.prod(shp))
        out[n + ".w"] = vec[o:o + k].reshape(shp).astype(np.float64)
        o += k
        nb = 1 if n == "head" else shp[-1]
        out[n + ".b"] = vec[o:o + nb].astype(np.float64)
        o += nb
    assert o == len(vec)
    return out


# ----------------------------------------------------------------- ops

def conv3(x, W, b):
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, Wd, W.shape[3])) + b
    for ky in range(3):
        for kx in range(3):
            out += xp[:, ky:ky + H, kx:kx + Wd, :] @ W[ky, kx]
    return out


def conv3_backward(x, W, g):
    """Gradients of conv3 wrt its input, weights and bias for the output
    gradient g."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            gxp[:, ky:ky + H, kx:kx + Wd, :] += g @ W[ky, kx].T
            gW[ky, kx] = np.einsum("bhwc,bhwd->cd", xp[:, ky:ky + H, kx:kx + Wd, :], g)
    return gxp[:, 1:-1, 1:-1, :], gW, g.sum(axis=(0, 1, 2))


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def upconv(x, U, b):
    B, H, W, _ = x.shape
    out = np.zeros((B, 2 * H, 2 * W, U.shape[3])) + b
    for dy in range(2):
        for dx in range(2):
            out[:, dy::2, dx::2, :] += x @ U[dy, dx]
    return out


def upconv_backward(x, U, g):
    gx = np.zeros_like(x)
    gU = np.zeros_like(U)
    for dy in range(2):
        for dx in range(2):
            gd = g[:, dy::2, dx::2, :]
            gx += gd @ U[dy, dx].T
            gU[dy, dx] = np.einsum("bhwc,bhwd->cd", x, gd)
    return gx, gU, g.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


# ------------------------------------------------------------- network

def forward(p: dict, x: np.ndarray):
    """Output y (batch, H, W) and the activations needed by backward."""
    a = {"x": x}
    a["e1a"] = relu(conv3(x, p["enc1a.w"], p["enc1a.b"]))
    a["s1"] = relu(conv3(a["e1a"], p["enc1b.w"], p["enc1b.b"]))
    a["p1"] = pool(a["s1"])
    a["e2a"] = relu(conv3(a["p1"], p["enc2a.w"], p["enc2a.b"]))
    a["s2"] = relu(conv3(a["e2a"], p["enc2b.w"], p["enc2b.b"]))
    a["p2"] = pool(a["s2"])
    a["e3a"] = relu(conv3(a["p2"], p["enc3a.w"], p["enc3a.b"]))
    a["s3"] = relu(conv3(a["e3a"], p["enc3b.w"], p["enc3b.b"]))
    a["p3"] = pool(a["s3"])
    a["e4a"] = relu(conv3(a["p3"], p["enc4a.w"], p["enc4a.b"]))
    a["e4b"] = relu(conv3(a["e4a"], p["enc4b.w"], p["enc4b.b"]))
    prev = a["e4b"]
    for k in (3, 2, 1):
        u = upconv(prev, p[f"up{k}.w"], p[f"up{k}.b"])
        a[f"c{k}"] = np.concatenate([u, a[f"s{k}"]], axis=3)
        a[f"d{k}a"] = relu(conv3(a[f"c{k}"], p[f"dec{k}a.w"], p[f"dec{k}a.b"]))
        a[f"d{k}b"] = relu(conv3(a[f"d{k}a"], p[f"dec{k}b.w"], p[f"dec{k}b.b"]))
        a[f"in_up{k}"] = prev
        prev = a[f"d{k}b"]
    y = a["d1b"] @ p["head.w"] + p["head.b"][0]
    return y, a


def loss(y, t):
    return 0.5 * np.sum((y - t) ** 2) / y.size


def backward(p: dict, a: dict, gy: np.ndarray):
    """Gradients of every parameter and of the input for the output
    gradient gy (batch, H, W)."""
    g = {}
    g["head.w"] = np.einsum("bhwc,bhw->c", a["d1b"], gy)
    g["head.b"] = np.array([gy.sum()])
    gpost = gy[..., None] * p["head.w"]            # wrt d1b
    up_grad = None
    for k in (1, 2, 3):
        gpre = gpost * (a[f"d{k}b"] > 0)
        gin, g[f"dec{k}b.w"], g[f"dec{k}b.b"] = conv3_backward(a[f"d{k}a"], p[f"dec{k}b.w"], gpre)
        gpre = gin * (a[f"d{k}a"] > 0)
        gc, g[f"dec{k}a.w"], g[f"dec{k}a.b"] = conv3_backward(a[f"c{k}"], p[f"dec{k}a.w"], gpre)
        nu = p[f"up{k}.w"].shape[3]
        g[f"skip{k}"] = gc[..., nu:]
        gprev, g[f"up{k}.w"], g[f"up{k}.b"] = upconv_backward(a[f"in_up{k}"], p[f"up{k}.w"],
                                                             gc[..., :nu])
        gpost = gprev   # wrt d{k+1}b, or e4b after k = 3
        up_grad = gprev
    gpre = up_grad * (a["e4b"] > 0)
    gin, g["enc4b.w"], g["enc4b.b"] = conv3_backward(a["e4a"], p["enc4b.w"], gpre)
    gpre = gin * (a["e4a"] > 0)
    gpool, g["enc4a.w"], g["enc4a.b"] = conv3_backward(a["p3"], p["enc4a.w"], gpre)
    for k in (3, 2, 1):
        gs = (g.pop(f"skip{k}") + pool_backward(gpool)) * (a[f"s{k}"] > 0)
        gin, g[f"enc{k}b.w"], g[f"enc{k}b.b"] = conv3_backward(a[f"e{k}a"], p[f"enc{k}b.w"], gs)
        gpre = gin * (a[f"e{k}a"] > 0)
        src = a["x"] if k == 1 else a[f"p{k - 1}"]
        gpool, g[f"enc{k}a.w"], g[f"enc{k}a.b"] = conv3_backward(src, p[f"enc{k}a.w"], gpre)
    g["x"] = gpool
    return g
