"""FP64 oracle of the warm-start network: a 4-level convolutional U-Net that
maps a channel's solid mask and Reynolds number to its steady (rho, u_x, u_y).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the slow, plainly
written statement that the CUDA network is checked against.  Nothing in the
package imports it.

The paper has no learned part; the network is the one the method's
acceleration plan names (4 levels, 32-256 channels, 3x3 kernels, trained on
steady fields the method generates).  Readings, all stated here once:

  layout       NCHW float64 arrays, batch first; an image is [H][W] = [ny][nx]
  conv3x3      y[n,o,i,j] = b[o] + sum_{c,di,dj} w[o,c,di,dj] x[n,c,i+di-1,j+dj-1],
               zero outside the image ("same" cross-correlation)
  level l      two conv3x3 + ReLU with C_l = base * 2^l channels (base 32)
  down         2x2 average pooling;  up: 2x nearest-neighbour repetition
  decoder      up(deeper) concatenated before the skip tensor, then two conv3x3 + ReLU
  head         1x1 conv (no ReLU) to 3 output channels
  inputs       channel 0: solid mask (1 solid, 0 fluid); channel 1: Re / 100;
               channels 2..7: zero (the kernels take 8 input channels)
  outputs      three channels: the scaled density deviation and velocity
  loss         mean over fluid nodes and the 3 channels of (out - target)^2
  optimizer    Adam with bias correction (beta1 0.9, beta2 0.999, eps 1e-8)

Every function is a direct loop or a NumPy contraction of its definition.
"""
from __future__ import annotations

import numpy as np

IN_CH = 8
OUT_CH = 3


def channels(levels: int = 4, base: int = 32) -> list[int]:
    return [base * (2 ** l) for l in range(levels)]


def layer_shapes(levels: int = 4, base: int = 32) -> list[tuple[str, int, int, int]]:
    """(name, c_out, c_in, k) of every conv, in parameter order."""
    ch = channels(levels, base)
    out = []
    cin = IN_CH
    for l, c in enumerate(ch):
        out.append((f"enc{l}a", c, cin, 3))
        out.append((f"enc{l}b", c, c, 3))
        cin = c
    for l in range(levels - 2, -1, -1):
        c = ch[l]
        out.append((f"dec{l}a", c, ch[l + 1] + c, 3))
        out.append((f"dec{l}b", c, c, 3))
    out.append(("head", OUT_CH, ch[0], 1))
    return out


def init_params(levels: int = 4, base: int = 32, seed: int = 0) -> dict:
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, co, ci, k in layer_shapes(levels, base):
        std = np.sqrt(2.0 / (ci * k * k))
        p[name + ".w"] = rng.normal(0.0, std, size=(co, ci, k, k))
        p[name + ".b"] = np.zeros(co)
    return p


# ------------------------------------------------------------- layers

def conv(x, w, b):
    """'same' cross-correlation of x [N][C][H][W] with w [O][C][k][k] (+ b)."""
    n, c, h, wd = x.shape
    o, c2, k, _ = w.shape
    assert c == c2
    r = k // 2
    xp = np.zeros((n, c, h + 2 * r, wd + 2 * r))
    xp[:, :, r:r + h, r:r + wd] = x
    y = np.zeros((n, o, h, wd))
    for di in range(k):
        for dj in range(k):
            patch = xp[:, :, di:di + h, dj:dj + wd]          # [N][C][H][W]
            y += np.einsum("nchw,oc->nohw", patch, w[:, :, di, dj])
    return y + b[None, :, None, None]


def conv_backward(x, w, dy):
    """Gradients of conv: (dx, dw, db) for the upstream gradient dy."""
    n, c, h, wd = x.shape
    o, _, k, _ = w.shape
    r = k // 2
    xp = np.zeros((n, c, h + 2 * r, wd + 2 * r))
    xp[:, :, r:r + h, r:r + wd] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(k):
        for dj in range(k):
            patch = xp[:, :, di:di + h, dj:dj + wd]
            dw[:, :, di, dj] = np.einsum("nohw,nchw->oc", dy, patch)
            dxp[:, :, di:di + h, dj:dj + wd] += np.einsum("nohw,oc->nchw", dy, w[:, :, di, dj])
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, r:r + h, r:r + wd], dw, db


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    """2x2 average pooling."""
    n, c, h, w = x.shape
    return x.reshape(n, c, h // 2, 2, w // 2, 2).mean(axis=(3, 5))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3) / 4.0


def up(x):
    """2x nearest-neighbour upsampling."""
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_backward(dy):
    n, c, h, w = dy.shape
    return dy.reshape(n, c, h // 2, 2, w // 2, 2).sum(axis=(3, 5))


# ------------------------------------------------------------ network

def forward(p: dict, x: np.ndarray, levels: int = 4, keep: bool = False):
    """Network output [N][3][H][W]; with keep, also the cache for backward.

    encoder level l:  in_l = x (l = 0) or pool(e_{l-1});
                      e_l = relu(conv_b(relu(conv_a(in_l))))
    decoder level l:  cat_l = [up(d_{l+1}), e_l] (d_{L-1} = e_{L-1});
                      d_l = relu(conv_b(relu(conv_a(cat_l))))
    head:             y = conv1x1(d_0)
    """
    cache = {"enc": [], "dec": {}}
    e = []
    for l in range(levels):
        inp = x if l == 0 else pool(e[-1])
        za = conv(inp, p[f"enc{l}a.w"], p[f"enc{l}a.b"])
        aa = relu(za)
        zb = conv(aa, p[f"enc{l}b.w"], p[f"enc{l}b.b"])
        e.append(relu(zb))
        cache["enc"].append((inp, za, aa, zb))
    d = e[-1]
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([up(d), e[l]], axis=1)
        za = conv(cat, p[f"dec{l}a.w"], p[f"dec{l}a.b"])
        aa = relu(za)
        zb = conv(aa, p[f"dec{l}b.w"], p[f"dec{l}b.b"])
        d = relu(zb)
        cache["dec"][l] = (cat, za, aa, zb)
    y = conv(d, p["head.w"], p["head.b"])
    cache["head"] = d
    return (y, cache) if keep else y


def backward(p: dict, cache, dy, levels: int = 4) -> dict:
    """Gradient of every parameter for the upstream gradient dy of the output."""
    g = {}
    dd, g["head.w"], g["head.b"] = conv_backward(cache["head"], p["head.w"], dy)
    dskip = {}
    for l in range(0, levels - 1):  # decoder levels in reverse order of the forward
        cat, za, aa, zb = cache["dec"][l]
        dzb = dd * (zb > 0)
        daa, g[f"dec{l}b.w"], g[f"dec{l}b.b"] = conv_backward(aa, p[f"dec{l}b.w"], dzb)
        dza = daa * (za > 0)
        dcat, g[f"dec{l}a.w"], g[f"dec{l}a.b"] = conv_backward(cat, p[f"dec{l}a.w"], dza)
        cu = cat.shape[1] - cache["enc"][l][3].shape[1]  # channels of up(d_{l+1})
        dskip[l] = dcat[:, cu:]
        dd = up_backward(dcat[:, :cu])  # gradient of d_{l+1}
    de = dd  # gradient of e_{L-1} = d_{L-1}
    for l in range(levels - 1, -1, -1):
        inp, za, aa, zb = cache["enc"][l]
        dzb = de * (zb > 0)
        daa, g[f"enc{l}b.w"], g[f"enc{l}b.b"] = conv_backward(aa, p[f"enc{l}b.w"], dzb)
        dza = daa * (za > 0)
        dinp, g[f"enc{l}a.w"], g[f"enc{l}a.b"] = conv_backward(inp, p[f"enc{l}a.w"], dza)
        if l > 0:
            de = pool_backward(dinp) + dskip[l - 1]
    return g


def loss(y, target, fluid):
    """Masked mean squared error and its gradient; fluid is [N][H][W] of 0/1."""
    m = fluid[:, None, :, :].astype(np.float64)
    cnt = m.sum() * y.shape[1]
    d = (y - target) * m
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def adam(p: dict, g: dict, state: dict, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state holds 't' and the moments."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
