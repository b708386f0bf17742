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

Every operation keeps the dtype of its inputs: FP64 arrays (the oracle)
give an FP64 network; FP32 arrays give the same network in plain FP32
arithmetic, which tells how far FP32 rounding alone moves a result.

``forward`` and ``backward`` take an optional rounding ``q`` applied where
a reduced-precision implementation stores values (the input, every stored
activation and activation gradient, the convolution weights): with
q = round_bf16 the ReLU decisions are taken on the same BF16 values as a
BF16 implementation takes them; q = None is the plain FP64 network.
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

def round_bf16(a):
    """Round to the nearest BF16 value (ties to even) through float32."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def _ident(a):
    return a


def conv3(x, W, b):
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, Wd, W.shape[3]), dtype=x.dtype) + b
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
    out = np.zeros((B, 2 * H, 2 * W, U.shape[3]), dtype=x.dtype) + b
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

def forward(p: dict, x: np.ndarray, q=None):
    """Output y (batch, H, W) and the activations needed by backward."""
    q = q or _ident
    a = {"x": q(x)}

    def cv(inp, name):
        return q(relu(conv3(inp, q(p[name + ".w"]), p[name + ".b"])))

    a["e1a"] = cv(a["x"], "enc1a")
    a["s1"] = cv(a["e1a"], "enc1b")
    a["p1"] = q(pool(a["s1"]))
    a["e2a"] = cv(a["p1"], "enc2a")
    a["s2"] = cv(a["e2a"], "enc2b")
    a["p2"] = q(pool(a["s2"]))
    a["e3a"] = cv(a["p2"], "enc3a")
    a["s3"] = cv(a["e3a"], "enc3b")
    a["p3"] = q(pool(a["s3"]))
    a["e4a"] = cv(a["p3"], "enc4a")
    a["e4b"] = cv(a["e4a"], "enc4b")
    prev = a["e4b"]
    for k in (3, 2, 1):
        u = q(upconv(prev, q(p[f"up{k}.w"]), p[f"up{k}.b"]))
        a[f"c{k}"] = np.concatenate([u, a[f"s{k}"]], axis=3)
        a[f"d{k}a"] = cv(a[f"c{k}"], f"dec{k}a")
        a[f"d{k}b"] = cv(a[f"d{k}a"], f"dec{k}b")
        a[f"in_up{k}"] = prev
        prev = a[f"d{k}b"]
    y = a["d1b"] @ p["head.w"] + p["head.b"][0]
    return y, a


def loss(y, t):
    return 0.5 * np.sum((y - t) ** 2) / y.size


def backward(p: dict, a: dict, gy: np.ndarray, q=None):
    """Gradients of every parameter and of the input for the output
    gradient gy (batch, H, W)."""
    q = q or _ident
    W = {k: (q(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in p.items()}
    g = {}
    g["head.w"] = np.einsum("bhwc,bhw->c", a["d1b"], gy)
    g["head.b"] = np.array([gy.sum()])
    gpre = q(gy[..., None] * p["head.w"] * (a["d1b"] > 0))   # wrt d1b, pre-activation
    for k in (1, 2, 3):
        gin, g[f"dec{k}b.w"], g[f"dec{k}b.b"] = conv3_backward(a[f"d{k}a"], W[f"dec{k}b.w"], gpre)
        gpre = q(gin * (a[f"d{k}a"] > 0))
        gc, g[f"dec{k}a.w"], g[f"dec{k}a.b"] = conv3_backward(a[f"c{k}"], W[f"dec{k}a.w"], gpre)
        gc = q(gc)
        nu = p[f"up{k}.w"].shape[3]
        g[f"skip{k}"] = gc[..., nu:]
        gprev, g[f"up{k}.w"], g[f"up{k}.b"] = upconv_backward(a[f"in_up{k}"], W[f"up{k}.w"],
                                                             gc[..., :nu])
        gpre = q(gprev * (a[f"in_up{k}"] > 0))   # pre-activation of d{k+1}b, or of e4b
    gin, g["enc4b.w"], g["enc4b.b"] = conv3_backward(a["e4a"], W["enc4b.w"], gpre)
    gpre = q(gin * (a["e4a"] > 0))
    gpool, g["enc4a.w"], g["enc4a.b"] = conv3_backward(a["p3"], W["enc4a.w"], gpre)
    gpool = q(gpool)
    for k in (3, 2, 1):
        gs = q((g.pop(f"skip{k}") + pool_backward(gpool)) * (a[f"s{k}"] > 0))
        gin, g[f"enc{k}b.w"], g[f"enc{k}b.b"] = conv3_backward(a[f"e{k}a"], W[f"enc{k}b.w"], gs)
        gpre = q(gin * (a[f"e{k}a"] > 0))
        src = a["x"] if k == 1 else a[f"p{k - 1}"]
        gpool, g[f"enc{k}a.w"], g[f"enc{k}a.b"] = conv3_backward(src, W[f"enc{k}a.w"], gpre)
        gpool = q(gpool)
    g["x"] = gpool
    return g


# ------------------------------------------------------------ optimiser

def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One step of Adam (Kingma and Ba, 2015, Algorithm 1) in FP64 at step
    number t >= 1: the moment estimates m <- beta1 m + (1 - beta1) g and
    v <- beta2 v + (1 - beta2) g^2, their bias-corrected values
    m / (1 - beta1^t) and v / (1 - beta2^t), and the update
    w <- w - lr mhat / (sqrt(vhat) + eps).  Returns the new (w, m, v)."""
    w, g, m, v = (np.asarray(a, dtype=np.float64) for a in (w, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v

