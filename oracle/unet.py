"""Learned warm start: a 3D U-Net on periodic voxel fields, FP64 reference.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Not in the paper: the
network proposes the fluctuation-strain increment that starts the Newton
iteration of an increment (Sect. 2.1 leaves the initial guess open).

Input (IN_CH = 32 channels per voxel): the grain's orientation quaternion
(4), its phase (1), the prescribed macroscopic increment direction (9), the
previous increment's normalised fluctuation increment (9) and that
increment's direction (9).  The network itself is generic in these
channels; what they hold matters only to the solver.

Tensors are (C, nz, ny, nx).  A convolution is periodic (indices wrap) with
3x3x3 taps: y[o, p] = b[o] + sum_{t, i} W[t, o, i] x[i, p + d_t], tap
t = 9 (dz+1) + 3 (dy+1) + (dx+1), d_t = (dz, dy, dx) in {-1, 0, 1}^3.
`bf16` rounds a tensor to bfloat16 (round to nearest even), used to mirror
the points where the GPU stores bfloat16.

Architecture (4 levels, channels 16, 32, 64, 64; leaky ReLU with slope
1/8 on the negative side after every 3x3x3 conv (plain ReLU let whole layers
die in training; the power of two keeps slope * bfloat16 exact); 2x2x2 average pooling down, nearest-neighbour upsampling up, skip
connections by channel concatenation; a 1x1x1 head to 9 outputs):
  e1 = c(c(x, 32->16), 16->16)          at n
  e2 = c(c(pool e1, 16->32), 32->32)    at n/2
  e3 = c(c(pool e2, 32->64), 64->64)    at n/4
  e4 = c(c(pool e3, 64->64), 64->64)    at n/8
  d3 = c(c([up e4, e3], 128->64), 64->64)
  d2 = c(c([up d3, e2], 96->32), 32->32)
  d1 = c(c([up d2, e1], 48->16), 16->16)
  y  = head(d1, 16->9)
"""

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]

LAYERS = [  # (name, cin, cout)
    ("e1a", 32, 16), ("e1b", 16, 16),
    ("e2a", 16, 32), ("e2b", 32, 32),
    ("e3a", 32, 64), ("e3b", 64, 64),
    ("e4a", 64, 64), ("e4b", 64, 64),
    ("d3a", 128, 64), ("d3b", 64, 64),
    ("d2a", 96, 32), ("d2b", 32, 32),
    ("d1a", 48, 16), ("d1b", 16, 16),
]
HEAD = ("head", 16, 9)
IN_CH = LAYERS[0][1]
SLOPE = 0.125  # leaky ReLU slope for z <= 0


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x, d):
    """x[..., p + d] with periodic wrap (d = (dz, dy, dx))."""
    return np.roll(x, shift=(-d[0], -d[1], -d[2]), axis=(-3, -2, -1))


def conv(x, W, b=None):
    """Periodic 3x3x3 convolution; W has shape (27, cout, cin)."""
    y = np.zeros((W.shape[1],) + x.shape[1:])
    for t, d in enumerate(TAPS):
        y += np.einsum("oi,i...->o...", W[t], shift(x, d))
    if b is not None:
        y += b[:, None, None, None]
    return y


def conv_grad_input(dy, W):
    """Adjoint of conv in x: dx[i, p] = sum_{t, o} W[t, o, i] dy[o, p - d_t]."""
    dx = np.zeros((W.shape[2],) + dy.shape[1:])
    for t, d in enumerate(TAPS):
        dx += np.einsum("oi,o...->i...", W[t], shift(dy, (-d[0], -d[1], -d[2])))
    return dx


def conv_grad_weight(x, dy):
    """dW[t, o, i] = sum_p dy[o, p] x[i, p + d_t]."""
    return np.stack([np.einsum("ozyx,izyx->oi", dy, shift(x, d)) for d in TAPS])


def pool(x):
    """2x2x2 average pooling."""
    c, nz, ny, nx = x.shape
    return x.reshape(c, nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(2, 4, 6))


def pool_grad(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_grad(dy):
    c, nz, ny, nx = dy.shape
    return dy.reshape(c, nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(2, 4, 6))


def init_params(seed=0):
    """He-uniform weights, zero biases (any initialisation serves the tests)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in LAYERS:
        lim = np.sqrt(6.0 / (27 * ci))
        p[name] = (rng.uniform(-lim, lim, (27, co, ci)), np.zeros(co))
    name, ci, co = HEAD
    lim = np.sqrt(6.0 / ci)
    p[name] = (rng.uniform(-lim, lim, (co, ci)), np.zeros(co))
    return p


def forward(p, x, round_bf16=False):
    """Network output (9, n, n, n) and the cache the backward pass needs.
    With round_bf16, weights and every stored activation are rounded to
    bfloat16 (accumulation stays FP64)."""
    R = bf16 if round_bf16 else (lambda a: a)
    cache = {"x": R(x)}

    def cr(name, a):
        W, b = p[name]
        z = conv(a, R(W), b)
        out = R(np.where(z > 0, z, SLOPE * z))
        cache[name] = (a, out)
        return out

    e1 = cr("e1b", cr("e1a", cache["x"]))
    e2 = cr("e2b", cr("e2a", R(pool(e1))))
    e3 = cr("e3b", cr("e3a", R(pool(e2))))
    e4 = cr("e4b", cr("e4a", R(pool(e3))))
    d3 = cr("d3b", cr("d3a", np.concatenate([up(e4), e3])))
    d2 = cr("d2b", cr("d2a", np.concatenate([up(d3), e2])))
    d1 = cr("d1b", cr("d1a", np.concatenate([up(d2), e1])))
    Wh, bh = p["head"]
    y = np.einsum("oi,i...->o...", R(Wh), d1) + bh[:, None, None, None]
    cache["d1"] = d1
    return y, cache


def backward(p, cache, dy, round_bf16=False):
    """Gradients of all parameters for the output gradient dy (9, n, n, n).
    With round_bf16, the activation gradients are rounded to bfloat16 where
    the GPU stores them."""
    R = bf16 if round_bf16 else (lambda a: a)
    g = {}
    Wh, bh = p["head"]
    d1 = cache["d1"]
    g["head"] = (np.einsum("ozyx,izyx->oi", dy, d1), dy.sum(axis=(1, 2, 3)))
    dd1 = R(np.einsum("oi,o...->i...", R(Wh), dy))

    def cb(name, da_out):
        a_in, out = cache[name]
        W, b = p[name]
        dz = da_out * np.where(out > 0, 1.0, SLOPE)
        g[name] = (conv_grad_weight(a_in, dz), dz.sum(axis=(1, 2, 3)))
        return R(conv_grad_input(dz, R(W)))

    def split(da, c1):
        return da[:c1], da[c1:]

    da = cb("d1a", cb("d1b", dd1))
    dup2, de1 = split(da, 32)
    da = cb("d2a", cb("d2b", R(up_grad(dup2))))
    dup3, de2 = split(da, 64)
    da = cb("d3a", cb("d3b", R(up_grad(dup3))))
    dup4, de3 = split(da, 64)
    de4 = cb("e4a", cb("e4b", R(up_grad(dup4))))
    de3 = R(de3 + pool_grad(de4))
    de3 = cb("e3a", cb("e3b", de3))
    de2 = R(de2 + pool_grad(de3))
    de2 = cb("e2a", cb("e2b", de2))
    de1 = R(de1 + pool_grad(de2))
    cb("e1a", cb("e1b", de1))
    return g


def mse(y, t):
    """Mean squared error over all elements and its gradient."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size
