"""Learned warm-start surrogate: a periodic convolutional U-Net of four levels
(32 to 128 channels) trained and run on the library's own BF16 tensor-core
kernels (include/lbm_surrogate.h).

Every operation of the forward pass, the backward pass and the Adam update is
one lbm_sg_* kernel launched through the C-ABI; PyTorch only provides device
memory (allocation and zero-fill) and the stream.

Network (all convolutions periodic 3x3; grids H, H/2, H/4, H/8 with H and W
multiples of 8; every channel count padded to a multiple of 16 with zero
weights that stay zero):
  e1   conv 4 -> 32, ReLU                      level 1: s1   (cat1[:, :32])
  pool 2x2, e2 conv 32 -> 64, ReLU             level 2: s2   (cat2[:, :64])
  pool 2x2, e3 conv 64 -> 128, ReLU            level 3: s3   (cat3[:, :128])
  pool 2x2, b  conv 128 -> 128, ReLU           level 4
  up x2 into cat3[:, 128:], d3 conv 256 -> 64, ReLU    level 3
  up x2 into cat2[:, 64:],  d2 conv 128 -> 32, ReLU    level 2
  up x2 into cat1[:, 32:],  d1 conv 64 -> 32, ReLU     level 1
  out  conv 32 -> 4                            delta
  result = in + delta, in = (phi, rho u_x, rho u_y, P) / scale
"""
import ctypes

import numpy as np

from . import lbm as L

LAYERS = [("e1", 4, 32), ("e2", 32, 64), ("e3", 64, 128), ("b", 128, 128),
          ("d3", 256, 64), ("d2", 128, 32), ("d1", 64, 32), ("out", 32, 4)]
POOL = 2      # pooling / upsampling factor between levels
LEVELS = 4
NC = 4        # real channels of the input and output: phi, rho u_x, rho u_y, P
CO_MAX = 128  # output channels one lbm_sg_conv3x3 call produces at most


def _pad16(c):
    return (c + 15) // 16 * 16


def init_params(seed=0):
    """He-normal weights (the last layer scaled by 0.1, so the map starts
    near the identity) and zero biases, real shapes W[co, ci, 3, 3], FP64."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co in LAYERS:
        std = np.sqrt(2.0 / (ci * 9)) * (0.1 if name == "out" else 1.0)
        params[name + ".W"] = rng.normal(0.0, std, size=(co, ci, 3, 3))
        params[name + ".b"] = np.zeros(co)
    return params


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _off(t, channels):
    """Address of channel `channels` of the first pixel of a channels-last tensor."""
    return ctypes.c_void_p(t.data_ptr() + channels * t.element_size())


def _ck(rc, what):
    if rc != L.OK:
        raise L.LbmError(rc, what)


class Surrogate:
    """Parameters, Adam state and activation buffers for batches of N images of
    H x W (multiples of 8, N H W / 64 a multiple of 16)."""

    def __init__(self, N, H, W, params=None, seed=0, stream=None):
        import torch
        self.torch = torch
        self.lib = L.load()
        f = POOL ** (LEVELS - 1)
        if H % f or W % f or (N * H * W // (f * f)) % 16:
            raise ValueError("H, W multiples of 8 and N H W / 64 a multiple of 16")
        self.N, self.H, self.W = N, H, W
        self.M = [N * H * W // (POOL ** (2 * l)) for l in range(LEVELS)]   # pixels per level
        self.HW = [(H // POOL ** l, W // POOL ** l) for l in range(LEVELS)]
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        dev = "cuda"
        f32, b16 = torch.float32, torch.bfloat16
        z = lambda *s, dt=f32: torch.zeros(*s, dtype=dt, device=dev)
        self.layers = {}
        for name, ci, co in LAYERS:
            cip, cop = _pad16(ci), _pad16(co)
            self.layers[name] = dict(ci=ci, co=co, cip=cip, cop=cop,
                                     W=z(cop, 9, cip), b=z(cop), W16=z(cop, 9, cip, dt=b16), Wt=z(cip, 9, cop, dt=b16),
                                     mW=z(cop, 9, cip), vW=z(cop, 9, cip), mb=z(cop), vb=z(cop),
                                     gW=z(cop, 9, cip), gb=z(cop))
        self.set_params(params if params is not None else init_params(seed))
        M1, M2, M3, M4 = self.M
        # forward activations: pre-activations (FP32) for the ReLU backward,
        # post-activations (bf16) as the next layer's input
        self.x16, self.x32 = z(M1, 16, dt=b16), z(M1, NC)
        self.a = {"e1": z(M1, 32), "e2": z(M2, 64), "e3": z(M3, 128), "b": z(M4, 128),
                  "d3": z(M3, 64), "d2": z(M2, 32), "d1": z(M1, 32)}
        self.cat1, self.cat2, self.cat3 = z(M1, 64, dt=b16), z(M2, 128, dt=b16), z(M3, 256, dt=b16)
        self.p1, self.p2, self.p3 = z(M2, 32, dt=b16), z(M3, 64, dt=b16), z(M4, 128, dt=b16)
        self.hb, self.h3, self.h2, self.h1 = z(M4, 128, dt=b16), z(M3, 64, dt=b16), z(M2, 32, dt=b16), z(M1, 32, dt=b16)
        self.delta = z(M1, 16)
        # backward buffers (FP32 gradients and their bf16 copies per level)
        self.g_delta, self.g16_1 = z(M1, 16), z(M1, 64, dt=b16)
        self.gc1, self.gs1, self.ga1 = z(M1, 64), z(M1, 32), z(M1, 32)
        self.gc2, self.gs2, self.ga2, self.g16_2 = z(M2, 128), z(M2, 64), z(M2, 64), z(M2, 64, dt=b16)
        self.gc3, self.gs3, self.ga3, self.g16_3 = z(M3, 256), z(M3, 128), z(M3, 128), z(M3, 128, dt=b16)
        self.gt2, self.gt3 = z(M2, 32), z(M3, 64)
        self.ghb, self.ga4, self.g16_4, self.gp3 = z(M4, 128), z(M4, 128), z(M4, 128, dt=b16), z(M4, 128)
        self.gp2, self.gp1, self.gpool = z(M3, 64), z(M2, 32), z(M1, 32)
        lib = self.lib
        scratch = max(lib.lbm_sg_wgrad_scratch_floats(N, H, W, 64, 32),
                      lib.lbm_sg_wgrad_scratch_floats(N, H, W, 16, 32),
                      lib.lbm_sg_wgrad_scratch_floats(N, H, W, 32, 16),
                      lib.lbm_sg_wgrad_scratch_floats(N, H // 2, W // 2, 128, 32),
                      lib.lbm_sg_wgrad_scratch_floats(N, H // 2, W // 2, 32, 64),
                      lib.lbm_sg_wgrad_scratch_floats(N, H // 4, W // 4, 256, 64),
                      lib.lbm_sg_wgrad_scratch_floats(N, H // 4, W // 4, 64, 128),
                      lib.lbm_sg_wgrad_scratch_floats(N, H // 8, W // 8, 128, 128), 64 * 256)
        self.scratch = z(int(scratch))
        self.mse_scratch = torch.zeros(256, dtype=torch.float64, device=dev)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        self.step_count = 0

    # ---------------------------------------------------------------- parameters
    def set_params(self, params):
        """Load real-shape parameters (W[co, ci, 3, 3], b[co]) into the padded
        FP32 masters and their bf16 copies; resets the Adam moments."""
        t = self.torch
        for name, ci, co in LAYERS:
            ly = self.layers[name]
            Wr = np.zeros((ly["cop"], 9, ly["cip"]), dtype=np.float32)
            Wr[:co, :, :ci] = np.transpose(params[name + ".W"].reshape(co, ci, 9), (0, 2, 1))
            br = np.zeros(ly["cop"], dtype=np.float32)
            br[:co] = params[name + ".b"]
            ly["W"].copy_(t.from_numpy(Wr))
            ly["b"].copy_(t.from_numpy(br))
            for k in ("mW", "vW", "mb", "vb"):
                ly[k].zero_()
            n = ly["cop"] * 9
            _ck(self.lib.lbm_sg_to_bf16(_ptr(ly["W"]), ly["cip"], _ptr(ly["W16"]), ly["cip"], n, ly["cip"],
                                        self.stream), "lbm_sg_to_bf16")
            self._flip(name)
        self.step_count = 0

    def _flip(self, name):
        ly = self.layers[name]
        _ck(self.lib.lbm_sg_weight_flip(_ptr(ly["W16"]), _ptr(ly["Wt"]), ly["cip"], ly["cop"], self.stream),
            "lbm_sg_weight_flip")

    def params(self):
        """Real-shape FP64 copies of the master parameters."""
        out = {}
        for name, ci, co in LAYERS:
            ly = self.layers[name]
            Wr = ly["W"].cpu().numpy().astype(np.float64)[:co, :, :ci]
            out[name + ".W"] = np.transpose(Wr, (0, 2, 1)).reshape(co, ci, 3, 3)
            out[name + ".b"] = ly["b"].cpu().numpy().astype(np.float64)[:co]
        return out

    def grads(self):
        """Real-shape FP64 copies of the last backward pass's gradients."""
        out = {}
        for name, ci, co in LAYERS:
            ly = self.layers[name]
            g = ly["gW"].cpu().numpy().astype(np.float64)[:co, :, :ci]
            out[name + ".W"] = np.transpose(g, (0, 2, 1)).reshape(co, ci, 3, 3)
            out[name + ".b"] = ly["gb"].cpu().numpy().astype(np.float64)[:co]
        return out

    # ---------------------------------------------------------------- primitives
    def _conv(self, name, x, csx, y, csy, level):
        ly = self.layers[name]
        h, w = self.HW[level]
        _ck(self.lib.lbm_sg_conv3x3(x, csx, _ptr(ly["W16"]), _ptr(ly["b"]), y, csy, self.N, h, w, ly["cip"],
                                    ly["cop"], self.stream), "lbm_sg_conv3x3")

    def _conv_input_grad(self, name, g16, csg, gx, csx, level):
        """gx = gradient w.r.t. the layer's input: the convolution of g with the
        flipped weights, in slices of at most CO_MAX output channels."""
        ly = self.layers[name]
        h, w = self.HW[level]
        cip, cop = ly["cip"], ly["cop"]
        for c0 in range(0, cip, CO_MAX):
            nco = min(CO_MAX, cip - c0)
            wt = ctypes.c_void_p(ly["Wt"].data_ptr() + c0 * 9 * cop * 2)
            out = ctypes.c_void_p(gx.data_ptr() + c0 * 4)
            _ck(self.lib.lbm_sg_conv3x3(g16, csg, wt, None, out, csx, self.N, h, w, cop, nco, self.stream),
                "lbm_sg_conv3x3")

    def _wgrad(self, name, x, csx, g16, csg, level):
        ly = self.layers[name]
        h, w = self.HW[level]
        _ck(self.lib.lbm_sg_conv3x3_wgrad(x, csx, g16, csg, _ptr(ly["gW"]), _ptr(self.scratch), self.scratch.numel(),
                                          self.N, h, w, ly["cip"], ly["cop"], self.stream), "lbm_sg_conv3x3_wgrad")

    def _bgrad(self, name, g, csg, level):
        ly = self.layers[name]
        _ck(self.lib.lbm_sg_bias_grad(g, csg, _ptr(ly["gb"]), _ptr(self.scratch), self.M[level], ly["cop"],
                                      self.stream), "lbm_sg_bias_grad")

    def _relu(self, a, csa, y, csy, level, C):
        _ck(self.lib.lbm_sg_relu(a, csa, y, csy, self.M[level], C, self.stream), "lbm_sg_relu")

    def _pool(self, x, csx, y, csy, level_fine, C):
        h, w = self.HW[level_fine]
        _ck(self.lib.lbm_sg_pool(x, csx, y, csy, self.N, h, w, C, POOL, self.stream), "lbm_sg_pool")

    def _up(self, x, csx, y, csy, level_fine, C):
        h, w = self.HW[level_fine]
        _ck(self.lib.lbm_sg_upsample(x, csx, y, csy, self.N, h, w, C, POOL, self.stream), "lbm_sg_upsample")

    def _up_bwd(self, g, csg, gx, csx, level_fine, C):
        h, w = self.HW[level_fine]
        _ck(self.lib.lbm_sg_upsample_bwd(g, csg, gx, csx, self.N, h, w, C, POOL, self.stream), "lbm_sg_upsample_bwd")

    def _pool_bwd(self, g, csg, gx, csx, level_fine, C):
        h, w = self.HW[level_fine]
        _ck(self.lib.lbm_sg_pool_bwd(g, csg, gx, csx, self.N, h, w, C, POOL, self.stream), "lbm_sg_pool_bwd")

    def _relu_bwd(self, g, csg, a, csa, ga, ga16, level, C):
        _ck(self.lib.lbm_sg_relu_bwd(g, csg, a, csa, ga, ga16, self.M[level], C, self.stream), "lbm_sg_relu_bwd")

    def _add(self, a, csa, b, csb, out, cso, level, C):
        _ck(self.lib.lbm_sg_add(a, csa, b, csb, out, cso, self.M[level], C, self.stream), "lbm_sg_add")

    # ---------------------------------------------------------------- passes
    def set_input(self, x32):
        """x32: (M, 4) float32 device tensor of normalised inputs; builds the
        padded bf16 copy."""
        if tuple(x32.shape) != tuple(self.x32.shape):
            raise ValueError(f"x32: shape {tuple(self.x32.shape)} required, got {tuple(x32.shape)}")
        self.x32.copy_(x32)
        _ck(self.lib.lbm_sg_to_bf16(_ptr(self.x32), NC, _ptr(self.x16), 16, self.M[0], NC, self.stream),
            "lbm_sg_to_bf16")

    def forward(self):
        """delta (M, 16) float32 for the current input; out = input + delta[:, :4]."""
        p, a = _ptr, self.a
        self._conv("e1", p(self.x16), 16, p(a["e1"]), 32, 0)
        self._relu(p(a["e1"]), 32, p(self.cat1), 64, 0, 32)                 # s1 -> cat1[:, :32]
        self._pool(p(self.cat1), 64, p(self.p1), 32, 0, 32)
        self._conv("e2", p(self.p1), 32, p(a["e2"]), 64, 1)
        self._relu(p(a["e2"]), 64, p(self.cat2), 128, 1, 64)                # s2 -> cat2[:, :64]
        self._pool(p(self.cat2), 128, p(self.p2), 64, 1, 64)
        self._conv("e3", p(self.p2), 64, p(a["e3"]), 128, 2)
        self._relu(p(a["e3"]), 128, p(self.cat3), 256, 2, 128)              # s3 -> cat3[:, :128]
        self._pool(p(self.cat3), 256, p(self.p3), 128, 2, 128)
        self._conv("b", p(self.p3), 128, p(a["b"]), 128, 3)
        self._relu(p(a["b"]), 128, p(self.hb), 128, 3, 128)
        self._up(p(self.hb), 128, _off(self.cat3, 128), 256, 2, 128)        # cat3[:, 128:]
        self._conv("d3", p(self.cat3), 256, p(a["d3"]), 64, 2)
        self._relu(p(a["d3"]), 64, p(self.h3), 64, 2, 64)
        self._up(p(self.h3), 64, _off(self.cat2, 64), 128, 1, 64)          # cat2[:, 64:]
        self._conv("d2", p(self.cat2), 128, p(a["d2"]), 32, 1)
        self._relu(p(a["d2"]), 32, p(self.h2), 32, 1, 32)
        self._up(p(self.h2), 32, _off(self.cat1, 32), 64, 0, 32)           # cat1[:, 32:]
        self._conv("d1", p(self.cat1), 64, p(a["d1"]), 32, 0)
        self._relu(p(a["d1"]), 32, p(self.h1), 32, 0, 32)
        self._conv("out", p(self.h1), 32, p(self.delta), 16, 0)
        return self.delta

    def backward(self, target32):
        """Loss (device FP64 scalar) and gradients of the MSE of out against
        target32 ((M, 4) float32)."""
        lib, s = self.lib, self.stream
        p, a = _ptr, self.a
        M1 = self.M[0]
        t = self.torch
        if not (isinstance(target32, t.Tensor) and target32.dtype == t.float32 and target32.is_cuda
                and target32.is_contiguous() and tuple(target32.shape) == (M1, NC)
                and target32.device == self.x32.device):
            # the loss kernel reads M x 4 floats from this pointer unchecked
            raise ValueError(f"target32: a contiguous float32 CUDA tensor of shape ({M1}, {NC}) on "
                             f"{self.x32.device} is required")
        _ck(lib.lbm_sg_mse(p(self.x32), NC, p(self.delta), 16, p(target32), NC, p(self.g_delta), p(self.mse_scratch),
                           p(self.loss_dev), M1, NC, s), "lbm_sg_mse")
        _ck(lib.lbm_sg_to_bf16(p(self.g_delta), 16, p(self.g16_1), 16, M1, 16, s), "lbm_sg_to_bf16")
        # out: input gradient -> gt1 (FP32, 32 channels, reusing gs1)
        self._wgrad("out", p(self.h1), 32, p(self.g16_1), 16, 0)
        self._bgrad("out", p(self.g_delta), 16, 0)
        self._conv_input_grad("out", p(self.g16_1), 16, self.gs1, 32, 0)
        # d1 (level 1): d cat1
        self._relu_bwd(p(self.gs1), 32, p(a["d1"]), 32, p(self.ga1), p(self.g16_1), 0, 32)
        self._wgrad("d1", p(self.cat1), 64, p(self.g16_1), 32, 0)
        self._bgrad("d1", p(self.ga1), 32, 0)
        self._conv_input_grad("d1", p(self.g16_1), 32, self.gc1, 64, 0)
        self._up_bwd(_off(self.gc1, 32), 64, p(self.gt2), 32, 0, 32)       # -> d h2 (level 2)
        # d2 (level 2): d cat2
        self._relu_bwd(p(self.gt2), 32, p(a["d2"]), 32, p(self.ga2), p(self.g16_2), 1, 32)
        self._wgrad("d2", p(self.cat2), 128, p(self.g16_2), 32, 1)
        self._bgrad("d2", p(self.ga2), 32, 1)
        self._conv_input_grad("d2", p(self.g16_2), 32, self.gc2, 128, 1)
        self._up_bwd(_off(self.gc2, 64), 128, p(self.gt3), 64, 1, 64)      # -> d h3 (level 3)
        # d3 (level 3): d cat3
        self._relu_bwd(p(self.gt3), 64, p(a["d3"]), 64, p(self.ga3), p(self.g16_3), 2, 64)
        self._wgrad("d3", p(self.cat3), 256, p(self.g16_3), 64, 2)
        self._bgrad("d3", p(self.ga3), 64, 2)
        self._conv_input_grad("d3", p(self.g16_3), 64, self.gc3, 256, 2)
        self._up_bwd(_off(self.gc3, 128), 256, p(self.ghb), 128, 2, 128)   # -> d hb (level 4)
        # b (level 4)
        self._relu_bwd(p(self.ghb), 128, p(a["b"]), 128, p(self.ga4), p(self.g16_4), 3, 128)
        self._wgrad("b", p(self.p3), 128, p(self.g16_4), 128, 3)
        self._bgrad("b", p(self.ga4), 128, 3)
        self._conv_input_grad("b", p(self.g16_4), 128, self.gp3, 128, 3)
        # s3 receives the skip (gc3[:, :128]) and the pooled path
        self._pool_bwd(p(self.gp3), 128, p(self.ga3), 128, 2, 128)
        self._add(p(self.gc3), 256, p(self.ga3), 128, p(self.gs3), 128, 2, 128)
        self._relu_bwd(p(self.gs3), 128, p(a["e3"]), 128, p(self.ga3), p(self.g16_3), 2, 128)
        self._wgrad("e3", p(self.p2), 64, p(self.g16_3), 128, 2)
        self._bgrad("e3", p(self.ga3), 128, 2)
        self._conv_input_grad("e3", p(self.g16_3), 128, self.gp2, 64, 2)
        # s2
        self._pool_bwd(p(self.gp2), 64, p(self.ga2), 64, 1, 64)
        self._add(p(self.gc2), 128, p(self.ga2), 64, p(self.gs2), 64, 1, 64)
        self._relu_bwd(p(self.gs2), 64, p(a["e2"]), 64, p(self.ga2), p(self.g16_2), 1, 64)
        self._wgrad("e2", p(self.p1), 32, p(self.g16_2), 64, 1)
        self._bgrad("e2", p(self.ga2), 64, 1)
        self._conv_input_grad("e2", p(self.g16_2), 64, self.gp1, 32, 1)
        # s1
        self._pool_bwd(p(self.gp1), 32, p(self.gpool), 32, 0, 32)
        self._add(p(self.gc1), 64, p(self.gpool), 32, p(self.gs1), 32, 0, 32)
        self._relu_bwd(p(self.gs1), 32, p(a["e1"]), 32, p(self.ga1), p(self.g16_1), 0, 32)
        self._wgrad("e1", p(self.x16), 16, p(self.g16_1), 32, 0)
        self._bgrad("e1", p(self.ga1), 32, 0)
        return self.loss_dev

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for name, _, _ in LAYERS:
            ly = self.layers[name]
            _ck(self.lib.lbm_sg_adam(_ptr(ly["W"]), _ptr(ly["mW"]), _ptr(ly["vW"]), _ptr(ly["gW"]), ly["W"].numel(),
                                     lr, b1, b2, eps, self.step_count, _ptr(ly["W16"]), self.stream), "lbm_sg_adam")
            _ck(self.lib.lbm_sg_adam(_ptr(ly["b"]), _ptr(ly["mb"]), _ptr(ly["vb"]), _ptr(ly["gb"]), ly["b"].numel(),
                                     lr, b1, b2, eps, self.step_count, None, self.stream), "lbm_sg_adam")
            self._flip(name)

    def train_step(self, x32, target32, lr=1e-3):
        self.set_input(x32)
        self.forward()
        loss = self.backward(target32)
        self.adam(lr)
        return loss

    def flops_per_image(self, backward=True):
        """Multiply-add FLOPs of the convolutions of one image (padded channel
        counts, as the kernels compute them): forward, and with `backward` the
        input- and weight-gradient convolutions too."""
        level = {"e1": 0, "e2": 1, "e3": 2, "b": 3, "d3": 2, "d2": 1, "d1": 0, "out": 0}
        tot = 0
        for name, _, _ in LAYERS:
            ly = self.layers[name]
            h, w = self.HW[level[name]]
            fwd = 2 * h * w * 9 * ly["cip"] * ly["cop"]
            tot += fwd * (3 if backward else 1)
        return tot
