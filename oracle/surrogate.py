"""Oracle of the learned warm-start network: a plain FP64 numpy forward and
backward pass of the convolutional surrogate.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the
CPU baseline of bench.py; the product path never calls it.

The paper has no network; this is the reference for the library's own
tensor-core kernels (lbm_sg_* in include/lbm_surrogate.h), written from the
definitions:

* periodic 3x3 convolution ("same" size, the LB domains are periodic):
  out[p, co] = b[co] + sum_{ci, dy, dx} W[co, ci, dy, dx] in[p + (dy - 1, dx - 1), ci]
  with p + offset wrapped on the grid;
* ReLU, 2x2 average pooling, nearest upsampling by 2, channel concatenation;
* the residual map out = in + net(in) on normalised fields.

Layout: one sample is an (H, W, C) array (channels last), a batch is
(N, H, W, C).  Weights W[co, ci, 3, 3], biases b[co].

Architecture: a U-Net of four levels (grids H, H/2, H/4, H/8; H and W
multiples of 8), 32 to 128 channels:
  e1:  conv 4 -> 32, ReLU                          level 1: s1
  pool, e2: conv 32 -> 64, ReLU                    level 2: s2
  pool, e3: conv 64 -> 128, ReLU                   level 3: s3
  pool, b:  conv 128 -> 128, ReLU                  level 4
  up, concat [s3, up] (256), d3: conv -> 64, ReLU  level 3
  up, concat [s2, up] (128), d2: conv -> 32, ReLU  level 2
  up, concat [s1, up] (64),  d1: conv -> 32, ReLU  level 1
  out: conv 32 -> 4                                (delta)
  result = in + delta
"""
import numpy as np

LAYERS = [("e1", 4, 32), ("e2", 32, 64), ("e3", 64, 128), ("b", 128, 128),
          ("d3", 256, 64), ("d2", 128, 32), ("d1", 64, 32), ("out", 32, 4)]
POOL = 2
LEVELS = 4


def init_params(seed=0):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co in LAYERS:
        std = np.sqrt(2.0 / (ci * 9))
        if name == "out":
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


def pool(x, f=POOL):
    """f x f block means."""
    N, H, W, C = x.shape
    return x.reshape(N, H // f, f, W // f, f, C).mean(axis=(2, 4))


def pool_backward(g, f=POOL):
    return np.repeat(np.repeat(g, f, axis=1), f, axis=2) / (f * f)


def upsample(x, f=POOL):
    """Nearest upsampling: every value repeated over an f x f block."""
    return np.repeat(np.repeat(x, f, axis=1), f, axis=2)


def upsample_backward(g, f=POOL):
    N, H, W, C = g.shape
    return g.reshape(N, H // f, f, W // f, f, C).sum(axis=(2, 4))


def forward(params, x):
    """Returns (output, cache) for input x (N, H, W, 4), H and W multiples of 8."""
    P = params
    c = {"x": x}

    def layer(name, inp):
        c[name + ".in"] = inp
        a = conv3x3(inp, P[name + ".W"], P[name + ".b"])
        c[name] = a
        return np.maximum(a, 0.0)

    s1 = layer("e1", x)
    s2 = layer("e2", pool(s1))
    s3 = layer("e3", pool(s2))
    hb = layer("b", pool(s3))
    t3 = layer("d3", np.concatenate([s3, upsample(hb)], axis=3))
    t2 = layer("d2", np.concatenate([s2, upsample(t3)], axis=3))
    t1 = layer("d1", np.concatenate([s1, upsample(t2)], axis=3))
    c["out.in"] = t1
    delta = conv3x3(t1, P["out.W"], P["out.b"])
    return x + delta, c


def loss(out, target):
    """Mean squared error over all elements."""
    return float(np.mean((out - target) ** 2))


def backward(params, cache, out, target):
    """Gradients of loss(out, target) with respect to every parameter."""
    P = params
    g = {}
    gout = 2.0 * (out - target) / out.size

    def layer_back(name, gy):
        """gy: gradient w.r.t. the layer's ReLU output; returns the gradient
        w.r.t. its input and stores the parameter gradients."""
        ga = gy * (cache[name] > 0)
        gi, g[name + ".W"], g[name + ".b"] = conv3x3_backward(cache[name + ".in"], P[name + ".W"], ga)
        return gi

    # out = x + conv(t1): the identity branch carries no parameters
    gt1, g["out.W"], g["out.b"] = conv3x3_backward(cache["out.in"], P["out.W"], gout)
    gc1 = layer_back("d1", gt1)
    n1 = P["e1.W"].shape[0]
    gs1, gt2 = gc1[..., :n1], upsample_backward(gc1[..., n1:])
    gc2 = layer_back("d2", gt2)
    n2 = P["e2.W"].shape[0]
    gs2, gt3 = gc2[..., :n2], upsample_backward(gc2[..., n2:])
    gc3 = layer_back("d3", gt3)
    n3 = P["e3.W"].shape[0]
    gs3, ghb = gc3[..., :n3], upsample_backward(gc3[..., n3:])
    gs3 = gs3 + pool_backward(layer_back("b", ghb))
    gs2 = gs2 + pool_backward(layer_back("e3", gs3))
    gs1 = gs1 + pool_backward(layer_back("e2", gs2))
    layer_back("e1", gs1)
    return g
