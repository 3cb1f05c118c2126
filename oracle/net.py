"""FP64 CPU reference of the seed network (test infrastructure only).

The seed network predicts an initial pressure P^0 for the solve from the
gradient field and the mask.  Its layers, written plainly in numpy for one
sample at a time, channels-last arrays of shape (D, H, W, C):

* conv3  3x3x3 convolution, stride 1, zero padding; weights (27, Cin, Cout),
         tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)
* down   2x2x2 convolution, stride 2; weights (8, Cin, Cout), tap = pz*4+py*2+px
* up     2x2x2 transposed convolution, stride 2; weights (8, Cin, Cout): the
         output voxel (2Z+pz, 2Y+py, 2X+px) = input (Z, Y, X) @ W[tap]
* conv1  1x1x1 convolution; weights (1, Cin, Cout)
* relu

Model (4 levels: full, 1/2, 1/4, 1/8 resolution; 16-64 channels; skip
connections by addition before the ReLU):

    e0  = relu(conv3(x, 4->16))
    e1  = relu(down(e0, 16->32));   e1b = relu(conv3(e1, 32->32))
    e2  = relu(down(e1b, 32->48));  e2b = relu(conv3(e2, 48->48))
    e3  = relu(down(e2b, 48->64))
    m   = relu(conv3(e3, 64->64));  m2  = relu(conv3(m, 64->64))
    u2  = relu(up(m2, 64->48) + e2b); u2b = relu(conv3(u2, 48->48))
    u1  = relu(up(u2b, 48->32) + e1b); u1b = relu(conv3(u1, 32->32))
    u0  = relu(up(u1b, 32->16) + e0)
    out = conv1(u0, 16->1)

Loss: mean over valid cells of ((out - mean out) - (y - mean y))^2, both
means over valid cells (pressure is defined up to a constant).

Every backward here is the plain chain rule of its forward; finite
differences pin them (tests/test_oracle_net.py).
"""
from __future__ import annotations

import numpy as np

# (name, kind, cin, cout, input, skip)
LAYERS = [
    ("e0", "conv3", 4, 16, "x", None),
    ("e1", "down", 16, 32, "e0", None),
    ("e1b", "conv3", 32, 32, "e1", None),
    ("e2", "down", 32, 48, "e1b", None),
    ("e2b", "conv3", 48, 48, "e2", None),
    ("e3", "down", 48, 64, "e2b", None),
    ("m", "conv3", 64, 64, "e3", None),
    ("m2", "conv3", 64, 64, "m", None),
    ("u2", "up", 64, 48, "m2", "e2b"),
    ("u2b", "conv3", 48, 48, "u2", None),
    ("u1", "up", 48, 32, "u2b", "e1b"),
    ("u1b", "conv3", 32, 32, "u1", None),
    ("u0", "up", 32, 16, "u1b", "e0"),
    ("out", "conv1", 16, 1, "u0", None),
]
TAPS = {"conv3": 27, "down": 8, "up": 8, "conv1": 1}


def init_params(seed=0, dtype=np.float64):
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, kind, cin, cout, _, _ in LAYERS:
        taps = TAPS[kind]
        fan_in = cin * (taps if kind != "up" else 1)
        std = np.sqrt(2.0 / fan_in) if kind != "conv1" else np.sqrt(1.0 / fan_in)
        params[name + ".w"] = (rng.normal(size=(taps, cin, cout)) * std).astype(dtype)
        params[name + ".b"] = np.zeros(cout, dtype=dtype)
    return params


def _offsets3():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(x, w, b):
    D, H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((D, H, W, w.shape[2])) + b
    for t, (dz, dy, dx) in enumerate(_offsets3()):
        y += xp[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] @ w[t]
    return y


def conv3_backward(x, w, dy):
    D, H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for t, (dz, dyy, dx) in enumerate(_offsets3()):
        sl = (slice(1 + dz, 1 + dz + D), slice(1 + dyy, 1 + dyy + H), slice(1 + dx, 1 + dx + W))
        dw[t] = np.einsum("zyxc,zyxo->co", xp[sl], dy)
        dxp[sl] += dy @ w[t].T
    return dxp[1:-1, 1:-1, 1:-1], dw, dy.sum(axis=(0, 1, 2))


def _par():
    return [(pz, py, px) for pz in (0, 1) for py in (0, 1) for px in (0, 1)]


def down(x, w, b):
    D, H, W, _ = x.shape
    y = np.zeros((D // 2, H // 2, W // 2, w.shape[2])) + b
    for t, (pz, py, px) in enumerate(_par()):
        y += x[pz::2, py::2, px::2] @ w[t]
    return y


def down_backward(x, w, dy):
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (pz, py, px) in enumerate(_par()):
        dw[t] = np.einsum("zyxc,zyxo->co", x[pz::2, py::2, px::2], dy)
        dx[pz::2, py::2, px::2] = dy @ w[t].T
    return dx, dw, dy.sum(axis=(0, 1, 2))


def up(x, w, b):
    D, H, W, _ = x.shape
    y = np.zeros((2 * D, 2 * H, 2 * W, w.shape[2]))
    for t, (pz, py, px) in enumerate(_par()):
        y[pz::2, py::2, px::2] = x @ w[t]
    return y + b


def up_backward(x, w, dy):
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (pz, py, px) in enumerate(_par()):
        g = dy[pz::2, py::2, px::2]
        dw[t] = np.einsum("zyxc,zyxo->co", x, g)
        dx += g @ w[t].T
    return dx, dw, dy.sum(axis=(0, 1, 2))


def conv1(x, w, b):
    return x @ w[0] + b


def conv1_backward(x, w, dy):
    return dy @ w[0].T, np.einsum("zyxc,zyxo->co", x, dy)[None], dy.sum(axis=(0, 1, 2))


_FWD = {"conv3": conv3, "down": down, "up": up, "conv1": conv1}
_BWD = {"conv3": conv3_backward, "down": down_backward, "up": up_backward, "conv1": conv1_backward}


def forward(params, x, store=None):
    """x: (D, H, W, 4).  Returns (output (D, H, W), cache of activations).
    ``store`` optionally quantises every stored activation (e.g. to the
    storage precision of an implementation being compared); the arithmetic
    stays FP64."""
    act = {"x": x}
    for name, kind, cin, cout, src, skip in LAYERS:
        pre = _FWD[kind](act[src], params[name + ".w"], params[name + ".b"])
        if skip is not None:
            pre = pre + act[skip]
        a = pre if name == "out" else np.maximum(pre, 0.0)
        act[name] = a if (store is None or name == "out") else store(a)
    return act["out"][..., 0], act


def loss(out, target, valid):
    """Masked, mean-removed MSE and its gradient with respect to out."""
    v = valid.astype(bool)
    n = v.sum()
    d = np.where(v, out - target, 0.0)
    dm = d[v].mean()
    e = np.where(v, d - dm, 0.0)
    L = float((e[v] ** 2).sum() / n)
    g = np.where(v, 2.0 * e / n, 0.0)  # the mean's own derivative cancels (sum e = 0)
    return L, g


def backward(params, act, dout, operand=None):
    """Gradients of every parameter given dL/d(out) of shape (D, H, W).
    ``operand`` optionally quantises the masked output gradient where it
    enters the weight and data products (the bias gradient and the skip paths
    use it unquantised); the arithmetic stays FP64."""
    grads = {}
    dact = {name: None for name, *_ in LAYERS}
    dact["out"] = dout[..., None]
    for name, kind, cin, cout, src, skip in reversed(LAYERS):
        g = dact[name]
        if g is None:
            continue
        if name != "out":
            g = g * (act[name] > 0)
        gq = g if operand is None else operand(g)
        dx, dw, _ = _BWD[kind](act[src], params[name + ".w"], gq)
        db = g.sum(axis=(0, 1, 2))
        grads[name + ".w"] = dw
        grads[name + ".b"] = db
        if src != "x":
            dact[src] = dx if dact[src] is None else dact[src] + dx
        if skip is not None:
            dact[skip] = g if dact[skip] is None else dact[skip] + g
    return grads


def features(grad, valid, spacing):
    """Network input from a gradient field: channels (fx, fy, fz) * h / s and
    the mask, s = h * RMS over valid cells of |grad|, so the problem's
    linearity in f is removed.  grad: (3, D, H, W).  Returns (x, s)."""
    v = valid.astype(bool)
    h = float(spacing)
    mag2 = (grad ** 2).sum(axis=0)
    s = h * np.sqrt(mag2[v].mean()) if v.any() else 1.0
    s = s if s > 0 else 1.0
    x = np.zeros(valid.shape + (4,))
    for a in range(3):
        x[..., a] = np.where(v, grad[a] * h / s, 0.0)
    x[..., 3] = v.astype(np.float64)
    return x, s
