"""Oracle of the learned warm-start network: a plain FP64 numpy forward and
backward pass of the small convolutional surrogate.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the
CPU baseline of bench.py; the product path never calls it.

The paper has no network; this is the reference for the library's own
tensor-core kernels (lbm_sg_* in include/lbm_surrogate.h), written from the
definitions:

* periodic 3x3 convolution ("same" size, the LB domains are periodic):
  out[p, co] = b[co] + sum_{ci, dy, dx} W[co, ci, dy, dx] in[p + (dy - 1, dx - 1), ci]
  with p + offset wrapped on the grid;
* ReLU, 8x8 average pooling, nearest upsampling by 8, channel concatenation;
* the residual map out = in + net(in) on normalised fields.

Layout: one sample is an (H, W, C) array (channels last), a batch is
(N, H, W, C).  Weights W[co, ci, 3, 3], biases b[co].

Architecture (channel counts):
  e1:  conv 4 -> 16, ReLU                  (full resolution, x1)
  pool 8x8                                 (coarse grid)
  c1:  conv 16 -> 32, ReLU
  c2:  conv 32 -> 32, ReLU
  c3:  conv 32 -> 32, ReLU
  c4:  conv 32 -> 16, ReLU
  up 8x nearest, concat [x1, up]  -> 32 channels
  d1:  conv 32 -> 16, ReLU
  d2:  conv 16 -> 4                        (delta)
  out = in + delta
"""
import numpy as np

LAYERS = [("e1", 4, 16), ("c1", 16, 32), ("c2", 32, 32), ("c3", 32, 32), ("c4", 32, 16),
          ("d1", 32, 16), ("d2", 16, 4)]
POOL = 8


def init_params(seed=0):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co in LAYERS:
        std = np.sqrt(2.0 / (ci * 9))
        if name == "d2":
            std *= 0.1   # start close to the identity map
        params[name + ".W"] = rng.normal(0.0, std, size=(co, ci, 3, 3))
        params[name + ".b"] = np.zeros(co)
    return params


def conv3x3(x, W, b):
    """Periodic 3x3 convolution, straight from the definition: (N, H, W, Ci) -> (N, H, W, Co)."""
    N, H, Wd, Ci = x.shape
    Co = W.shape[0]
    out = np.broadcast_to(b, (N, H, Wd, Co)).copy()
    for dy in range(3):
        for dx in range(3):
            # value at p + (dy - 1, dx - 1): roll the grid by the opposite offset
            xs = np.roll(x, shift=(1 - dy, 1 - dx), axis=(1, 2))
            out += np.einsum("nhwi,oi->nhwo", xs, W[:, :, dy, dx])
    return out


def conv3x3_backward(x, W, gout):
    """Gradients of conv3x3 with respect to x, W and b."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            xs = np.roll(x, shift=(1 - dy, 1 - dx), axis=(1, 2))
            gW[:, :, dy, dx] = np.einsum("nhwo,nhwi->oi", gout, xs)
            # out[p] uses x[p + d]: x[q] receives gout[q - d]
            gx += np.roll(np.einsum("nhwo,oi->nhwi", gout, W[:, :, dy, dx]), shift=(dy - 1, dx - 1), axis=(1, 2))
    gb = gout.sum(axis=(0, 1, 2))
    return gx, gW, gb


def pool(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // POOL, POOL, W // POOL, POOL, C).mean(axis=(2, 4))


def pool_backward(g, shape):
    return np.repeat(np.repeat(g, POOL, axis=1), POOL, axis=2) / (POOL * POOL)


def upsample(x):
    return np.repeat(np.repeat(x, POOL, axis=1), POOL, axis=2)


def upsample_backward(g):
    N, H, W, C = g.shape
    return g.reshape(N, H // POOL, POOL, W // POOL, POOL, C).sum(axis=(2, 4))


def forward(params, x):
    """Returns (output, cache) for input x (N, H, W, 4), H and W multiples of 8."""
    c = {"x": x}
    P = params
    a = conv3x3(x, P["e1.W"], P["e1.b"]); c["e1"] = a; x1 = np.maximum(a, 0.0); c["x1"] = x1
    h = pool(x1); c["pool"] = h
    for name in ("c1", "c2", "c3", "c4"):
        c[name + ".in"] = h
        a = conv3x3(h, P[name + ".W"], P[name + ".b"]); c[name] = a
        h = np.maximum(a, 0.0)
    up = upsample(h)
    cat = np.concatenate([x1, up], axis=3); c["cat"] = cat
    a = conv3x3(cat, P["d1.W"], P["d1.b"]); c["d1"] = a; hd = np.maximum(a, 0.0); c["hd"] = hd
    delta = conv3x3(hd, P["d2.W"], P["d2.b"])
    return x + delta, c


def loss(out, target):
    """Mean squared error over all elements."""
    return float(np.mean((out - target) ** 2))


def backward(params, cache, out, target):
    """Gradients of loss(out, target) with respect to every parameter."""
    P = params
    g = {}
    gout = 2.0 * (out - target) / out.size
    # out = x + d2(hd): the identity branch carries no parameters
    ghd, g["d2.W"], g["d2.b"] = conv3x3_backward(cache["hd"], P["d2.W"], gout)
    ga = ghd * (cache["d1"] > 0)
    gcat, g["d1.W"], g["d1.b"] = conv3x3_backward(cache["cat"], P["d1.W"], ga)
    n1 = cache["x1"].shape[3]
    gx1 = gcat[..., :n1]
    gh = upsample_backward(gcat[..., n1:])
    for name in ("c4", "c3", "c2", "c1"):
        ga = gh * (cache[name] > 0)
        gh, g[name + ".W"], g[name + ".b"] = conv3x3_backward(cache[name + ".in"], P[name + ".W"], ga)
    gx1 = gx1 + pool_backward(gh, cache["x1"].shape)
    ga = gx1 * (cache["e1"] > 0)
    _, g["e1.W"], g["e1.b"] = conv3x3_backward(cache["x"], P["e1.W"], ga)
    return g
