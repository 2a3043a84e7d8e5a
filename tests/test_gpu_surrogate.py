"""The surrogate's tensor-core kernels against the FP64 oracle of the network
(oracle/surrogate.py).

* Exactness of the implicit-GEMM convolution, its weight gradient and the
  flipped-weight input gradient: with small integers every bf16 operand and
  every FP32 partial sum is exact, so the kernels must equal the oracle
  bit for bit (any fragment-layout slip shows here).
* The whole network, forward and backward, on random data: the oracle is
  given the same bf16-rounded weights; the GPU also rounds activations and
  gradients to bf16 between layers (8-bit mantissa), so the bound is a few
  2^-8 relative: 3e-2 normwise on the output delta, 6e-2 on each gradient.
* Training on the GPU lowers the loss.
"""
import ctypes

import numpy as np
import pytest

from oracle import surrogate as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00118_gb300 import build, lbm as L
    from paper_1812_00118_gb300 import surrogate as S
    build.build()
    L.load()
    return torch, L, S


def bf16_round(a):
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def nwise(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_conv_kernels_exact_on_integers(env):
    torch, L, S = env
    lib = L.load()
    rng = np.random.default_rng(0)
    N, H, W, Ci, Co = 2, 8, 24, 32, 48
    x = rng.integers(-3, 4, size=(N, H, W, Ci)).astype(np.float64)
    w = rng.integers(-3, 4, size=(Co, Ci, 3, 3)).astype(np.float64)
    b = rng.integers(-5, 6, size=Co).astype(np.float64)
    gy = rng.integers(-2, 3, size=(N, H, W, Co)).astype(np.float64)
    dev = "cuda"
    x16 = torch.tensor(x.reshape(-1, Ci), dtype=torch.bfloat16, device=dev)
    w16 = torch.tensor(np.transpose(w.reshape(Co, Ci, 9), (0, 2, 1)).copy(), dtype=torch.bfloat16, device=dev)
    bias = torch.tensor(b, dtype=torch.float32, device=dev)
    y = torch.zeros(N * H * W, Co, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.lbm_sg_conv3x3(ptr(x16), Ci, ptr(w16), ptr(bias), ptr(y), Co, N, H, W, Ci, Co, s) == 0
    ref = OS.conv3x3(x, w, b)
    assert np.array_equal(y.cpu().numpy().astype(np.float64), ref.reshape(-1, Co))
    # weight gradient
    g16 = torch.tensor(gy.reshape(-1, Co), dtype=torch.bfloat16, device=dev)
    gw = torch.zeros(Co, 9, Ci, dtype=torch.float32, device=dev)
    nscr = lib.lbm_sg_wgrad_scratch_floats(N, H, W, Ci, Co)
    scr = torch.zeros(nscr, dtype=torch.float32, device=dev)
    assert lib.lbm_sg_conv3x3_wgrad(ptr(x16), Ci, ptr(g16), Co, ptr(gw), ptr(scr), nscr, N, H, W, Ci, Co, s) == 0
    gx_ref, gw_ref, gb_ref = OS.conv3x3_backward(x, w, gy)
    got = np.transpose(gw.cpu().numpy().astype(np.float64), (0, 2, 1)).reshape(Co, Ci, 3, 3)
    assert np.array_equal(got, gw_ref)
    # input gradient through the flipped weights
    wt = torch.zeros(Ci, 9, Co, dtype=torch.bfloat16, device=dev)
    assert lib.lbm_sg_weight_flip(ptr(w16), ptr(wt), Ci, Co, s) == 0
    gx = torch.zeros(N * H * W, Ci, dtype=torch.float32, device=dev)
    assert lib.lbm_sg_conv3x3(ptr(g16), Co, ptr(wt), None, ptr(gx), Ci, N, H, W, Co, Ci, s) == 0
    assert np.array_equal(gx.cpu().numpy().astype(np.float64), gx_ref.reshape(-1, Ci))
    # bias gradient
    g32 = torch.tensor(gy.reshape(-1, Co), dtype=torch.float32, device=dev)
    gb = torch.zeros(Co, dtype=torch.float32, device=dev)
    assert lib.lbm_sg_bias_grad(ptr(g32), Co, ptr(gb), ptr(scr), N * H * W, Co, s) == 0
    assert np.array_equal(gb.cpu().numpy().astype(np.float64), gb_ref)


@pytest.mark.parametrize("N,H,W,Ci,Co", [(1, 2, 128, 16, 32), (2, 5, 128, 128, 32), (1, 7, 256, 32, 128),
                                         (3, 4, 256, 64, 48), (1, 64, 128, 32, 64), (1, 6, 128, 128, 128),
                                         (2, 3, 64, 32, 16), (2, 3, 64, 256, 64), (1, 4, 32, 128, 128)],
                         ids=["h2", "ci128", "co128", "co48", "rows1", "fallback", "w64", "ci256", "w32"])
def test_conv_row_march_exact_on_integers(env, N, H, W, Ci, Co):
    """Images whose width is a multiple of 128 go through the row-march
    convolution (its strip of input rows and all nine taps' weights in
    shared memory; the 128 x 128-channel case is too large for that and
    takes the tap kernel, as do the 64- and 32-wide images), with chunks of
    one row up to several per CTA; widths that are multiples of 32 take the
    row-march weight gradient (tcgen05 GEMMs over pixels, operands transposed
    in shared memory; 256 input channels in two blocks of 128).  On small
    integers every product and partial sum is exact: the
    results equal the oracle bit for bit, forward, through the flipped
    weights (the input gradient) and for the weight gradient."""
    torch, L, S = env
    lib = L.load()
    rng = np.random.default_rng(N * 1000 + H * 10 + Ci + Co)
    x = rng.integers(-3, 4, size=(N, H, W, Ci)).astype(np.float64)
    w = rng.integers(-3, 4, size=(Co, Ci, 3, 3)).astype(np.float64)
    b = rng.integers(-5, 6, size=Co).astype(np.float64)
    gy = rng.integers(-2, 3, size=(N, H, W, Co)).astype(np.float64)
    dev = "cuda"
    x16 = torch.tensor(x.reshape(-1, Ci), dtype=torch.bfloat16, device=dev)
    w16 = torch.tensor(np.transpose(w.reshape(Co, Ci, 9), (0, 2, 1)).copy(), dtype=torch.bfloat16, device=dev)
    bias = torch.tensor(b, dtype=torch.float32, device=dev)
    y = torch.zeros(N * H * W, Co, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.lbm_sg_conv3x3(ptr(x16), Ci, ptr(w16), ptr(bias), ptr(y), Co, N, H, W, Ci, Co, s) == 0
    assert np.array_equal(y.cpu().numpy().astype(np.float64), OS.conv3x3(x, w, b).reshape(-1, Co))
    wt = torch.zeros(Ci, 9, Co, dtype=torch.bfloat16, device=dev)
    assert lib.lbm_sg_weight_flip(ptr(w16), ptr(wt), Ci, Co, s) == 0
    g16 = torch.tensor(gy.reshape(-1, Co), dtype=torch.bfloat16, device=dev)
    gx = torch.zeros(N * H * W, Ci, dtype=torch.float32, device=dev)
    for c0 in range(0, Ci, 128):   # at most 128 output channels per call, as the network slices them
        nco = min(128, Ci - c0)
        wt_c = ctypes.c_void_p(wt.data_ptr() + c0 * 9 * Co * 2)
        gx_c = ctypes.c_void_p(gx.data_ptr() + c0 * 4)
        assert lib.lbm_sg_conv3x3(ptr(g16), Co, wt_c, None, gx_c, Ci, N, H, W, Co, nco, s) == 0
    gx_ref, gw_ref, _ = OS.conv3x3_backward(x, w, gy)
    assert np.array_equal(gx.cpu().numpy().astype(np.float64), gx_ref.reshape(-1, Ci))
    gw = torch.zeros(Co, 9, Ci, dtype=torch.float32, device=dev)
    nscr = lib.lbm_sg_wgrad_scratch_floats(N, H, W, Ci, Co)
    scr = torch.full((nscr,), float("nan"), dtype=torch.float32, device=dev)   # every partial must be written
    assert lib.lbm_sg_conv3x3_wgrad(ptr(x16), Ci, ptr(g16), Co, ptr(gw), ptr(scr), nscr, N, H, W, Ci, Co, s) == 0
    got = np.transpose(gw.cpu().numpy().astype(np.float64), (0, 2, 1)).reshape(Co, Ci, 3, 3)
    assert np.array_equal(got, gw_ref)
    assert lib.lbm_sg_status(s) == 0


def test_conv_rejects_bad_sizes(env):
    torch, L, S = env
    lib = L.load()
    t = torch.zeros(64, 16, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(64, 16, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.lbm_sg_conv3x3(ptr(t), 16, ptr(t), None, ptr(y), 16, 1, 8, 8, 12, 16, s) == L.EINVAL  # Ci % 16
    assert lib.lbm_sg_conv3x3(ptr(t), 16, ptr(t), None, ptr(y), 16, 1, 5, 3, 16, 16, s) == L.EINVAL  # pixels % 16
    assert lib.lbm_sg_conv3x3(None, 16, ptr(t), None, ptr(y), 16, 1, 8, 8, 16, 16, s) == L.EINVAL


def network_case(torch, S, seed=1, N=2, H=32, W=32):
    rng = np.random.default_rng(seed)
    P = S.init_params(seed)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.normal(scale=0.05, size=P[k].shape)
    x = rng.normal(size=(N, H, W, 4)).astype(np.float32)
    t = (x + 0.3 * rng.normal(size=x.shape)).astype(np.float32)
    sg = S.Surrogate(N, H, W, params=P)
    Pb = {k: (bf16_round(v) if k.endswith(".W") else v.astype(np.float32).astype(np.float64)) for k, v in P.items()}
    return sg, Pb, x, t


def test_network_forward_and_gradients_match_oracle(env):
    torch, L, S = env
    sg, Pb, x, t = network_case(torch, S)
    sg.set_input(torch.from_numpy(x.reshape(-1, 4)).cuda())
    delta = sg.forward()
    loss = sg.backward(torch.from_numpy(t.reshape(-1, 4)).cuda())
    torch.cuda.synchronize()
    xo = bf16_round(x)   # the network reads bf16 inputs; the residual adds the FP32 input
    out_o, cache = OS.forward(Pb, xo)
    delta_o = out_o - xo
    d = delta.cpu().numpy()[:, :4].reshape(delta_o.shape)
    assert nwise(d, delta_o) < 3e-2
    out_ref = x.astype(np.float64) + delta_o
    g_o = OS.backward(Pb, cache, out_ref, t.astype(np.float64))
    assert float(loss.item()) == pytest.approx(OS.loss(out_ref, t), rel=2e-2)
    g = sg.grads()
    for k in g_o:
        assert nwise(g[k], g_o[k]) < 6e-2, k


def test_training_lowers_the_loss(env):
    torch, L, S = env
    sg, _, x, t = network_case(torch, S, seed=2)
    xd = torch.from_numpy(x.reshape(-1, 4)).cuda()
    td = torch.from_numpy(t.reshape(-1, 4)).cuda()
    first = float(sg.train_step(xd, td, lr=2e-3).item())
    for _ in range(60):
        last = sg.train_step(xd, td, lr=2e-3)
    assert float(last.item()) < 0.7 * first


def test_phi_projection_and_phase_pressure(env):
    """lbm_sg_phi_project against its definition written out in numpy (the
    predicted change of phi kept to the start's interface band, clipped to
    [0, 1], the total of the start restored by moving the interfaces), and
    lbm_sg_phase_pressure against numpy means over the bulk phases."""
    torch, L, S = env
    lib = L.load()
    from paper_1812_00118_gb300 import inputs as I
    rng = np.random.default_rng(11)
    phi0, _, _ = I.sphere((1, 96, 96), (47.3, 48.6, 0), 20.0, 4.0, drop=True)
    phi0 = phi0.reshape(-1)
    pred = phi0 + rng.normal(scale=0.01, size=phi0.size)
    n = phi0.size
    d0 = torch.from_numpy(phi0).cuda()
    dp = torch.from_numpy(pred).cuda()
    scr = torch.zeros(1024, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.lbm_sg_phi_project(ptr(dp), ptr(d0), n, ptr(scr), s) == 0
    got = dp.cpu().numpy()
    m = 4 * phi0 * (1 - phi0)
    ref = np.clip(phi0 + m * (pred - phi0), 0.0, 1.0)
    wref = 4 * ref * (1 - ref)
    ref = ref + (phi0.sum() - ref.sum()) / wref.sum() * wref
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    assert abs(got.sum() - phi0.sum()) < 1e-10 * phi0.sum()
    bulk = (phi0 == 0.0) | (phi0 == 1.0)
    assert bulk.any() and np.array_equal(got[bulk], phi0[bulk])
    # bulk pressures
    P = rng.normal(size=n)
    dP = torch.from_numpy(P).cuda()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert lib.lbm_sg_phase_pressure(ptr(d0), ptr(dP), n, 0.01, ptr(out), ptr(scr), s) == 0
    o = out.cpu().numpy()
    hv, lt = phi0 >= 0.99, phi0 <= 0.01
    np.testing.assert_allclose(o, [P[hv].mean(), P[lt].mean(), hv.sum(), lt.sum()], rtol=1e-12)
    assert lib.lbm_sg_status(s) == 0
