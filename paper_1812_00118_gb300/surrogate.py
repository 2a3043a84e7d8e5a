"""Learned warm-start surrogate: a small periodic conv U-Net trained and run on
the library's own BF16 tensor-core kernels (include/lbm_surrogate.h).

Every operation of the forward pass, the backward pass and the Adam update is
one lbm_sg_* kernel launched through the C-ABI; PyTorch only provides device
memory (allocation and zero-fill) and the stream.

Network (channels; all convolutions periodic 3x3, every channel count padded
to a multiple of 16 with zero weights that stay zero):
  e1   conv 4 -> 16, ReLU              full resolution: x1
  pool 8 x 8 average
  c1   conv 16 -> 32, ReLU             coarse grid
  c2   conv 32 -> 32, ReLU
  c3   conv 32 -> 32, ReLU
  c4   conv 32 -> 16, ReLU
  up   8 x nearest, concatenated after x1 (32 channels)
  d1   conv 32 -> 16, ReLU
  d2   conv 16 -> 4                    delta
  out  = in + delta, in = (phi, ux, uy, P) / scale
"""
import ctypes

import numpy as np

from . import lbm as L

LAYERS = [("e1", 4, 16), ("c1", 16, 32), ("c2", 32, 32), ("c3", 32, 32), ("c4", 32, 16),
          ("d1", 32, 16), ("d2", 16, 4)]
POOL = 8
NC = 4   # real channels of the input and output: phi, ux, uy, P


def _pad16(c):
    return (c + 15) // 16 * 16


def init_params(seed=0):
    """He-normal weights (the last layer scaled by 0.1, so the map starts
    near the identity) and zero biases, real shapes W[co, ci, 3, 3], FP64."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co in LAYERS:
        std = np.sqrt(2.0 / (ci * 9)) * (0.1 if name == "d2" else 1.0)
        params[name + ".W"] = rng.normal(0.0, std, size=(co, ci, 3, 3))
        params[name + ".b"] = np.zeros(co)
    return params


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


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
        if H % POOL or W % POOL or (N * H * W // (POOL * POOL)) % 16:
            raise ValueError("H, W multiples of 8 and N H W / 64 a multiple of 16")
        self.N, self.H, self.W = N, H, W
        self.M = N * H * W
        self.Mc = self.M // (POOL * POOL)
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
        M, Mc = self.M, self.Mc
        self.x16, self.x32 = z(M, 16, dt=b16), z(M, NC)
        self.a_e1, self.cat16 = z(M, 16), z(M, 32, dt=b16)
        self.p16 = z(Mc, 16, dt=b16)
        self.a_c, self.h_c = {}, {}
        for name in ("c1", "c2", "c3", "c4"):
            co = self.layers[name]["cop"]
            self.a_c[name], self.h_c[name] = z(Mc, co), z(Mc, co, dt=b16)
        self.a_d1, self.hd = z(M, 16), z(M, 16, dt=b16)
        self.delta = z(M, 16)
        # backward buffers
        self.g_delta, self.g16 = z(M, 32), z(M, 32, dt=b16)
        self.gf_full, self.ga_full = z(M, 32), z(M, 32)
        self.gf_c, self.ga_c, self.ga16_c = z(Mc, 32), z(Mc, 32), z(Mc, 32, dt=b16)
        self.g_pool, self.g_x1 = z(M, 16), z(M, 16)
        scratch = max(self.lib.lbm_sg_wgrad_scratch_floats(N, H, W, 32, 32),
                      self.lib.lbm_sg_wgrad_scratch_floats(N, H // POOL, W // POOL, 32, 32), 64 * 32)
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

    # ---------------------------------------------------------------- passes
    def _conv(self, name, x, csx, y, csy, N, H, W, flip=False):
        ly = self.layers[name]
        if flip:   # input gradient: Ci and Co exchanged, no bias
            _ck(self.lib.lbm_sg_conv3x3(x, csx, _ptr(ly["Wt"]), None, y, csy, N, H, W, ly["cop"], ly["cip"],
                                        self.stream), "lbm_sg_conv3x3")
        else:
            _ck(self.lib.lbm_sg_conv3x3(x, csx, _ptr(ly["W16"]), _ptr(ly["b"]), y, csy, N, H, W, ly["cip"],
                                        ly["cop"], self.stream), "lbm_sg_conv3x3")

    def set_input(self, x32):
        """x32: (M, 4) float32 device tensor of normalised inputs; builds the
        padded bf16 copy."""
        self.x32.copy_(x32)
        _ck(self.lib.lbm_sg_to_bf16(_ptr(self.x32), NC, _ptr(self.x16), 16, self.M, NC, self.stream),
            "lbm_sg_to_bf16")

    def forward(self):
        """delta (M, 16) float32 for the current input; out = input + delta[:, :4]."""
        lib, s, N, H, W = self.lib, self.stream, self.N, self.H, self.W
        Hc, Wc = H // POOL, W // POOL
        M, Mc = self.M, self.Mc
        p = _ptr
        self._conv("e1", p(self.x16), 16, p(self.a_e1), 16, N, H, W)
        _ck(lib.lbm_sg_relu(p(self.a_e1), 16, p(self.cat16), 32, M, 16, s), "relu")            # x1 -> cat[:, :16]
        _ck(lib.lbm_sg_pool(p(self.cat16), 32, p(self.p16), 16, N, H, W, 16, s), "pool")
        h, ch = self.p16, 16
        for name in ("c1", "c2", "c3", "c4"):
            co = self.layers[name]["cop"]
            self._conv(name, p(h), ch, p(self.a_c[name]), co, N, Hc, Wc)
            _ck(lib.lbm_sg_relu(p(self.a_c[name]), co, p(self.h_c[name]), co, Mc, co, s), "relu")
            h, ch = self.h_c[name], co
        up = ctypes.c_void_p(self.cat16.data_ptr() + 16 * 2)                                    # cat[:, 16:]
        _ck(lib.lbm_sg_upsample(p(h), 16, up, 32, N, H, W, 16, s), "upsample")
        self._conv("d1", p(self.cat16), 32, p(self.a_d1), 16, N, H, W)
        _ck(lib.lbm_sg_relu(p(self.a_d1), 16, p(self.hd), 16, M, 16, s), "relu")
        self._conv("d2", p(self.hd), 16, p(self.delta), 16, N, H, W)
        return self.delta

    def _wgrad(self, name, x, csx, gy16, csg, N, H, W):
        ly = self.layers[name]
        _ck(self.lib.lbm_sg_conv3x3_wgrad(x, csx, gy16, csg, _ptr(ly["gW"]), _ptr(self.scratch), self.scratch.numel(),
                                          N, H, W, ly["cip"], ly["cop"], self.stream), "lbm_sg_conv3x3_wgrad")

    def _bgrad(self, name, g, csg, npix):
        ly = self.layers[name]
        _ck(self.lib.lbm_sg_bias_grad(g, csg, _ptr(ly["gb"]), _ptr(self.scratch), npix, ly["cop"], self.stream),
            "lbm_sg_bias_grad")

    def backward(self, target32):
        """Loss (device FP64 scalar) and gradients of the MSE of out against
        target32 ((M, 4) float32)."""
        lib, s, N, H, W = self.lib, self.stream, self.N, self.H, self.W
        Hc, Wc = H // POOL, W // POOL
        M, Mc = self.M, self.Mc
        p = _ptr
        _ck(lib.lbm_sg_mse(p(self.x32), NC, p(self.delta), 16, p(target32), NC, p(self.g_delta), p(self.mse_scratch),
                           p(self.loss_dev), M, NC, s), "lbm_sg_mse")
        _ck(lib.lbm_sg_to_bf16(p(self.g_delta), 16, p(self.g16), 16, M, 16, s), "to_bf16")
        # d2
        self._wgrad("d2", p(self.hd), 16, p(self.g16), 16, N, H, W)
        self._bgrad("d2", p(self.g_delta), 16, M)
        self._conv("d2", p(self.g16), 16, p(self.gf_full), 16, N, H, W, flip=True)      # g wrt hd
        # d1
        _ck(lib.lbm_sg_relu_bwd(p(self.gf_full), 16, p(self.a_d1), 16, p(self.ga_full), p(self.g16), M, 16, s), "relu_bwd")
        self._wgrad("d1", p(self.cat16), 32, p(self.g16), 16, N, H, W)
        self._bgrad("d1", p(self.ga_full), 16, M)
        self._conv("d1", p(self.g16), 16, p(self.gf_full), 32, N, H, W, flip=True)      # g wrt cat (32 ch)
        # coarse path: upsample backward of cat[:, 16:]
        g_up = ctypes.c_void_p(self.gf_full.data_ptr() + 16 * 4)
        _ck(lib.lbm_sg_upsample_bwd(g_up, 32, p(self.gf_c), 16, N, H, W, 16, s), "upsample_bwd")
        gin, cin = self.gf_c, 16
        prev = {"c4": "c3", "c3": "c2", "c2": "c1", "c1": None}
        for name in ("c4", "c3", "c2", "c1"):
            ly = self.layers[name]
            co, ci = ly["cop"], ly["cip"]
            _ck(lib.lbm_sg_relu_bwd(p(gin), cin, p(self.a_c[name]), co, p(self.ga_c), p(self.ga16_c), Mc, co, s),
                "relu_bwd")
            xin = self.h_c[prev[name]] if prev[name] else self.p16
            self._wgrad(name, p(xin), ci, p(self.ga16_c), co, N, Hc, Wc)
            self._bgrad(name, p(self.ga_c), co, Mc)
            self._conv(name, p(self.ga16_c), co, p(self.gf_c), ci, N, Hc, Wc, flip=True)
            gin, cin = self.gf_c, ci
        # x1 receives the pooled path and the skip
        _ck(lib.lbm_sg_pool_bwd(p(gin), 16, p(self.g_pool), 16, N, H, W, 16, s), "pool_bwd")
        _ck(lib.lbm_sg_add(p(self.gf_full), 32, p(self.g_pool), 16, p(self.g_x1), 16, M, 16, s), "add")
        _ck(lib.lbm_sg_relu_bwd(p(self.g_x1), 16, p(self.a_e1), 16, p(self.ga_full), p(self.g16), M, 16, s), "relu_bwd")
        self._wgrad("e1", p(self.x16), 16, p(self.g16), 16, N, H, W)
        self._bgrad("e1", p(self.ga_full), 16, M)
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
