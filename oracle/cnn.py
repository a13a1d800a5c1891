"""FP64 forward and backward of the warm-start U-Net (not a paper component; the learned
warm start is an addition to the method). Plain numpy, manual backpropagation.

Network (levels L, channels C, one input and one output channel, periodic 3x3 convolutions):
  encoder level 0:      a = relu(conv(u)),  e_0 = relu(conv(a))                (1 -> C -> C)
  encoder level l > 0:  p = avgpool2(e_{l-1}); a = relu(conv(p)); e_l = relu(conv(a))
  decoder level l = L-2 ... 0 (d_{L-1} = e_{L-1}):
                        s = up2(d_{l+1}) + e_l; a = relu(conv(s)); d_l = relu(conv(a))
  output:               v = u + conv(d_0)                                       (C -> 1)
conv(x)[co, y, x] = b[co] + sum_{ci, ky, kx} W[co, ci, ky, kx] x[ci, (y+ky-1) mod H, (x+kx-1) mod W]
avgpool2 averages 2 x 2 blocks; up2 repeats every value on a 2 x 2 block.
Loss: mean over all elements of (v - target)^2.

Parameters are listed in a fixed order (see `param_shapes`); the CUDA library uses the same
order and the same [C_out][C_in][3][3] weight layout for its flat parameter vector.

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

import numpy as np


def param_shapes(levels: int = 4, channels: int = 32) -> list[tuple[str, tuple]]:
    C = channels
    shapes = [("in.W", (C, 1, 3, 3)), ("in.b", (C,)), ("e0.W", (C, C, 3, 3)), ("e0.b", (C,))]
    for l in range(1, levels):
        shapes += [(f"e{l}a.W", (C, C, 3, 3)), (f"e{l}a.b", (C,)), (f"e{l}b.W", (C, C, 3, 3)), (f"e{l}b.b", (C,))]
    for l in range(levels - 2, -1, -1):
        shapes += [(f"d{l}a.W", (C, C, 3, 3)), (f"d{l}a.b", (C,)), (f"d{l}b.W", (C, C, 3, 3)), (f"d{l}b.b", (C,))]
    shapes += [("out.W", (1, C, 3, 3)), ("out.b", (1,))]
    return shapes


def init_params(levels: int = 4, channels: int = 32, seed: int = 0, out_scale: float = 0.1) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes(levels, channels):
        if name.endswith(".W"):
            fan_in = shp[1] * 9
            std = np.sqrt(2.0 / fan_in) * (out_scale if name.startswith("out") else 1.0)
            p[name] = rng.standard_normal(shp) * std
        else:
            p[name] = np.zeros(shp)
    return p


def flatten(p: dict, levels: int, channels: int) -> np.ndarray:
    return np.concatenate([p[n].ravel() for n, _ in param_shapes(levels, channels)])


def unflatten(v: np.ndarray, levels: int, channels: int) -> dict:
    out, o = {}, 0
    for n, shp in param_shapes(levels, channels):
        k = int(np.prod(shp))
        out[n] = v[o:o + k].reshape(shp).astype(np.float64)
        o += k
    return out


# ---------------------------------------------------------------------------------------
# layers
# ---------------------------------------------------------------------------------------

def _shift(x, ky, kx):
    """x[..., y + ky - 1, x + kx - 1] with periodic indices."""
    return np.roll(x, (-(ky - 1), -(kx - 1)), axis=(2, 3))


def conv(x, W, b):
    out = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, ky, kx], _shift(x, ky, kx))
    return out + b[None, :, None, None]


def conv_backward(x, W, dout, dx_store=None):
    """(dx, dW, db) of conv(x, W, b) given d(out). `dx_store`, if given, is applied to d(out)
    where it enters dx and dW (not db), for convolutions with at least two input and two
    output channels: it lets a test evaluate those gradients from a d(out) held in a lower
    precision, as an implementation that stores it that way for those products does."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    dxo = dout if dx_store is None or min(W.shape[0], W.shape[1]) < 2 else dx_store(dout)
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dxo, _shift(x, ky, kx))
            dx += np.roll(np.einsum("oc,bohw->bchw", W[:, :, ky, kx], dxo), (ky - 1, kx - 1), axis=(2, 3))
    return dx, dW, dout.sum(axis=(0, 2, 3))


def avgpool2(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def avgpool2_backward(d):
    return np.repeat(np.repeat(d, 2, axis=2), 2, axis=3) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_backward(d):
    B, C, H, W = d.shape
    return d.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


# ---------------------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------------------

def forward(p: dict, u: np.ndarray, levels: int, store=None):
    """u: [B, H, W] -> (v [B, H, W], cache).

    `store`, if given, is applied to every intermediate feature map as it is stored (all of
    them except the input u and the output v); it lets a test evaluate the network with
    feature maps held in a lower precision, so that ReLU decisions are taken on the same
    values as in an implementation that stores them that way. None keeps FP64."""
    S = (lambda t: t) if store is None else store
    x = u[:, None, :, :].astype(np.float64)
    cache = {"u": x}
    enc = []
    for l in range(levels):
        if l == 0:
            inp = x
            wa, ba, wb, bb = p["in.W"], p["in.b"], p["e0.W"], p["e0.b"]
        else:
            inp = S(avgpool2(enc[-1]))
            wa, ba, wb, bb = p[f"e{l}a.W"], p[f"e{l}a.b"], p[f"e{l}b.W"], p[f"e{l}b.b"]
        a = S(np.maximum(conv(inp, wa, ba), 0.0))
        e = S(np.maximum(conv(a, wb, bb), 0.0))
        cache[f"enc{l}"] = (inp, a, e)
        enc.append(e)
    d = enc[-1]
    for l in range(levels - 2, -1, -1):
        s = S(up2(d) + enc[l])
        a = S(np.maximum(conv(s, p[f"d{l}a.W"], p[f"d{l}a.b"]), 0.0))
        d = S(np.maximum(conv(a, p[f"d{l}b.W"], p[f"d{l}b.b"]), 0.0))
        cache[f"dec{l}"] = (s, a, d)
    v = x + conv(d, p["out.W"], p["out.b"])
    cache["d0"] = d
    return v[:, 0], cache


def backward(p: dict, cache: dict, dv: np.ndarray, levels: int, gstore=None) -> dict:
    """Gradients of every parameter given d(loss)/dv ([B, 1, H, W]); `gstore` is passed to
    conv_backward as dx_store."""
    g = {}
    cb = lambda x, W, d: conv_backward(x, W, d, gstore)  # noqa: E731
    dd, g["out.W"], g["out.b"] = cb(cache["d0"], p["out.W"], dv)
    denc = [np.zeros_like(cache[f"enc{l}"][2]) for l in range(levels)]
    # decoder, from the output back to the bottom: level 0, 1, ..., L-2
    for l in range(0, levels - 1):
        s, a, d = cache[f"dec{l}"]
        dz = dd * (d > 0)
        da, g[f"d{l}b.W"], g[f"d{l}b.b"] = cb(a, p[f"d{l}b.W"], dz)
        dz = da * (a > 0)
        ds, g[f"d{l}a.W"], g[f"d{l}a.b"] = cb(s, p[f"d{l}a.W"], dz)
        denc[l] += ds                 # s = up2(d_{l+1}) + e_l
        dd = up2_backward(ds)         # into d_{l+1}
    denc[levels - 1] += dd            # d_{L-1} = e_{L-1}
    # encoder, from the bottom up to level 0
    for l in range(levels - 1, -1, -1):
        inp, a, e = cache[f"enc{l}"]
        names = ("in", "e0") if l == 0 else (f"e{l}a", f"e{l}b")
        dz = denc[l] * (e > 0)
        da, g[f"{names[1]}.W"], g[f"{names[1]}.b"] = cb(a, p[f"{names[1]}.W"], dz)
        dz = da * (a > 0)
        dinp, g[f"{names[0]}.W"], g[f"{names[0]}.b"] = cb(inp, p[f"{names[0]}.W"], dz)
        if l > 0:
            denc[l - 1] += avgpool2_backward(dinp)
    return g


def loss_and_grads(p: dict, u: np.ndarray, target: np.ndarray, levels: int, store=None, gstore=None):
    """MSE loss (mean over every element) and its parameter gradients (`store` as in forward,
    `gstore` as in backward)."""
    v, cache = forward(p, u, levels, store)
    diff = v - target
    loss = float(np.mean(diff * diff))
    dv = 2.0 * diff / diff.size
    return loss, backward(p, cache, dv[:, None, :, :], levels, gstore), v
