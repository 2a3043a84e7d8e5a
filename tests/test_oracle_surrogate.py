"""Pins of the surrogate network oracle (oracle/surrogate.py) against what
the definitions fix: a brute-force loop convolution, the response to a unit
impulse, adjoint identities of pooling and upsampling, the identity map when
the last layer is zero, and central finite differences of the loss for
every parameter tensor of the four-level U-Net."""
import numpy as np
import pytest

from oracle import surrogate as S


def conv_brute(x, W, b):
    N, H, Wd, Ci = x.shape
    Co = W.shape[0]
    out = np.zeros((N, H, Wd, Co))
    for n in range(N):
        for y in range(H):
            for xx in range(Wd):
                for co in range(Co):
                    acc = b[co]
                    for ci in range(Ci):
                        for dy in range(3):
                            for dx in range(3):
                                acc += W[co, ci, dy, dx] * x[n, (y + dy - 1) % H, (xx + dx - 1) % Wd, ci]
                    out[n, y, xx, co] = acc
    return out


def test_conv_matches_loop_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 7, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    np.testing.assert_allclose(S.conv3x3(x, W, b), conv_brute(x, W, b), rtol=0, atol=1e-12)


def test_conv_impulse_response():
    # a unit value at (y0, x0, ci) reaches out[(y0 - dy + 1), (x0 - dx + 1), co] with weight W[co, ci, dy, dx]
    rng = np.random.default_rng(1)
    W = rng.normal(size=(2, 3, 3, 3))
    b = np.array([0.5, -0.25])
    x = np.zeros((1, 6, 6, 3))
    y0, x0, ci = 2, 3, 1
    x[0, y0, x0, ci] = 1.0
    out = S.conv3x3(x, W, b)
    for dy in range(3):
        for dx in range(3):
            np.testing.assert_allclose(out[0, (y0 - dy + 1) % 6, (x0 - dx + 1) % 6], W[:, ci, dy, dx] + b, atol=1e-15)
    assert np.allclose(out[0, 5, 0], b)   # untouched pixel


@pytest.mark.parametrize("f", [2, 8])
def test_pool_and_upsample_adjoints(f):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 16, 24, 3))
    y = rng.normal(size=(2, 16 // f, 24 // f, 3))
    assert np.isclose(np.sum(S.pool(x, f) * y), np.sum(x * S.pool_backward(y, f)))
    assert np.isclose(np.sum(S.upsample(y, f) * x), np.sum(y * S.upsample_backward(x, f)))
    np.testing.assert_allclose(S.pool(S.upsample(y, f), f), y)
    # a block mean by hand
    np.testing.assert_allclose(S.pool(x, f)[1, 1, 2, 0], x[1, f:2 * f, 2 * f:3 * f, 0].mean())


def test_identity_when_last_layer_is_zero():
    rng = np.random.default_rng(3)
    P = S.init_params(3)
    P["out.W"][:] = 0.0
    P["out.b"][:] = 0.0
    x = rng.normal(size=(1, 16, 16, 4))
    out, _ = S.forward(P, x)
    assert np.array_equal(out, x)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 4, 5, 2))
    W = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    gout = rng.normal(size=(1, 4, 5, 3))
    f = lambda x_, W_, b_: float(np.sum(S.conv3x3(x_, W_, b_) * gout))
    gx, gW, gb = S.conv3x3_backward(x, W, gout)
    e = 1e-6
    for arr, grad, args in ((x, gx, 0), (W, gW, 1), (b, gb, 2)):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            ap, am = arr.copy(), arr.copy()
            ap[idx] += e
            am[idx] -= e
            vals = [x, W, b]
            vals[args] = ap
            fp = f(*vals)
            vals[args] = am
            fm = f(*vals)
            assert (fp - fm) / (2 * e) == pytest.approx(grad[idx], rel=1e-6, abs=1e-9)


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(5)
    P = S.init_params(5)
    for k in P:   # biases away from zero so that ReLU kinks are not hit by the probes
        if k.endswith(".b"):
            P[k] = rng.normal(scale=0.1, size=P[k].shape)
    x = rng.normal(size=(2, 16, 16, 4))
    t = rng.normal(size=(2, 16, 16, 4))
    out, cache = S.forward(P, x)
    g = S.backward(P, cache, out, t)
    # every layer and the skip paths carry gradient
    assert all(np.abs(g[k]).max() > 0 for k in g)
    e = 1e-6
    for name in P:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += e
            Pm[name][idx] -= e
            fd = (S.loss(S.forward(Pp, x)[0], t) - S.loss(S.forward(Pm, x)[0], t)) / (2 * e)
            # abs: the rounding of the two losses (~2e-16 of a loss of ~2)
            # divided by the step 2e-6
            assert fd == pytest.approx(g[name][idx], rel=1e-5, abs=1e-9), (name, idx)
