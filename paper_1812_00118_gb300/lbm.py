"""ctypes binding of liblbm (include/lbm.h): argument marshalling only.

Every call goes straight to the C-ABI of the CUDA library; no step of the
method runs in Python.  Fields may be numpy float64 arrays (host) or torch
float64 CUDA tensors (device); populations and fields are laid out as the
header describes (x fastest, vectors component-major).

If liblbm.so has not been built (``paper_1812_00118_gb300.build``), loading
raises ``LbmLibraryMissing``: there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_CHECKED=1 in the environment selects the checked debugging build
# (paper_1812_00118_gb300.build.build(checked=True)); it must exist.
LIB_PATH = os.path.join(_PKG, "_lib", "liblbm_checked.so" if os.environ.get("LBM_CHECKED") == "1" else "liblbm.so")

D2Q9, D3Q19 = 0, 1
PERIODIC, WALL = 0, 1
F64, F32, F16S, BF16S = 0, 1, 2, 3
STORE_NAMES = {F64: "f64", F32: "f32", F16S: "f16s", BF16S: "bf16s"}

OK, EINVAL, ENOMEM, ECUDA, EDIVERGED, ETIMEOUT, ENOTSUP, ECHECKED = 0, -1, -2, -3, -4, -5, -6, -7
INIT_NONEQ = 1
CREATE_GHOST_BAND = 1


class LbmLibraryMissing(RuntimeError):
    pass


class LbmError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int * 3)]


class lbm_params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double), ("W", ctypes.c_double), ("sigma", ctypes.c_double),
                ("rho_L", ctypes.c_double), ("rho_H", ctypes.c_double),
                ("nu_L", ctypes.c_double), ("nu_H", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("force_mode", ctypes.c_int),
                ("eps", ctypes.c_double), ("hocorr", ctypes.c_int), ("store", ctypes.c_int),
                ("P_ref", ctypes.c_double), ("g_scale", ctypes.c_double),
                ("C_dtheta", ctypes.c_double)]


_lib = None

# (name, restype, argtypes) of every symbol include/lbm.h declares
_VP, _DP, _IP = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
SIGNATURES = [
    ("lbm_create", ctypes.c_int, [ctypes.POINTER(lbm_grid), ctypes.c_int, ctypes.POINTER(lbm_params), _VP,
                                  ctypes.POINTER(_VP)]),
    ("lbm_create_ex", ctypes.c_int, [ctypes.POINTER(lbm_grid), ctypes.c_int, ctypes.POINTER(lbm_params), _VP,
                                     ctypes.c_int, ctypes.POINTER(_VP)]),
    ("lbm_layout", ctypes.c_int, [ctypes.POINTER(lbm_grid), ctypes.c_int, ctypes.POINTER(lbm_params), ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_longlong)]),
    ("lbm_init_fields", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    ("lbm_init_fields_ex", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int]),
    ("lbm_step", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_step_profiled", ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    ("lbm_macro", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    ("lbm_get_populations", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    ("lbm_set_populations", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    ("lbm_diagnostics", ctypes.c_int, [_VP, _DP]),
    ("lbm_laplace", ctypes.c_int, [_VP, _DP, ctypes.c_double, ctypes.c_double, _DP]),
    ("lbm_lattice_info", ctypes.c_int, [ctypes.c_int, _IP, _IP, _DP]),
    ("lbm_launch_count", ctypes.c_longlong, [_VP]),
    ("lbm_stream", _VP, [_VP]),
    ("lbm_set_wall_velocity", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _DP]),
    ("lbm_set_phi_correction", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_set_wait_limit", ctypes.c_int, [_VP, ctypes.c_longlong]),
    ("lbm_set_tile", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    ("lbm_get_tile", ctypes.c_int, [_VP, _IP, _IP, _IP, _IP]),
    ("lbm_autotune", ctypes.c_int, [_VP, ctypes.c_int, _IP, _IP, _DP]),
    ("lbm_field_sums_noalloc", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_longlong, ctypes.c_double,
                                              ctypes.c_double, _VP, _VP]),
    ("lbm_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_params), _VP,
                                        ctypes.POINTER(_VP)]),
    ("lbm_batch_grid", _VP, [_VP, ctypes.c_int]),
    ("lbm_batch_step", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_batch_step_sequential", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_batch_set_tile", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    ("lbm_batch_get_tile", ctypes.c_int, [_VP, _IP, _IP, _IP, _IP]),
    ("lbm_batch_set_graph", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_batch_autotune", ctypes.c_int, [_VP, ctypes.c_int, _IP, _IP, _DP]),
    ("lbm_batch_launch_count", ctypes.c_longlong, [_VP]),
    ("lbm_batch_plan", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lbm_grid), ctypes.c_int, ctypes.c_int, _IP,
                                      ctypes.c_int]),
    ("lbm_batch_destroy", None, [_VP]),
    ("lbm_sg_conv3x3", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_int] + [ctypes.c_int] * 5 + [_VP]),
    ("lbm_sg_wgrad_scratch_floats", ctypes.c_longlong, [ctypes.c_int] * 5),
    ("lbm_sg_conv3x3_wgrad", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, ctypes.c_longlong]
     + [ctypes.c_int] * 5 + [_VP]),
    ("lbm_sg_weight_flip", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("lbm_sg_bias_grad", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_longlong, ctypes.c_int, _VP]),
    ("lbm_sg_relu", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, _VP]),
    ("lbm_sg_relu_bwd", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, ctypes.c_longlong,
                                       ctypes.c_int, _VP]),
    ("lbm_sg_to_bf16", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, _VP]),
    ("lbm_checked_status", ctypes.c_int, [_VP]),
    ("lbm_is_checked_build", ctypes.c_int, []),
    ("lbm_sg_status", ctypes.c_int, [_VP]),
    ("lbm_sg_add", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_longlong,
                                  ctypes.c_int, _VP]),
    ("lbm_sg_pool", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int] + [ctypes.c_int] * 5 + [_VP]),
    ("lbm_sg_pool_bwd", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int] + [ctypes.c_int] * 5 + [_VP]),
    ("lbm_sg_upsample", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int] + [ctypes.c_int] * 5 + [_VP]),
    ("lbm_sg_upsample_bwd", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int] + [ctypes.c_int] * 5 + [_VP]),
    ("lbm_sg_mse", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP,
                                  ctypes.c_longlong, ctypes.c_int, _VP]),
    ("lbm_sg_adam", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_longlong, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_int, _VP, _VP]),
    ("lbm_sg_pack", ctypes.c_int, [_VP, _VP, _VP, _VP, _DP, _VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_longlong,
                                   _VP]),
    ("lbm_sg_unpack", ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _DP, ctypes.c_double,
                                     ctypes.c_double, _VP, ctypes.c_longlong, _VP]),
    ("lbm_sg_residual", ctypes.c_int, [_VP, _VP, ctypes.c_longlong, _VP, _VP, _VP]),
    ("lbm_sg_smooth", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     _VP]),
    ("lbm_sg_phi_project", ctypes.c_int, [_VP, _VP, ctypes.c_longlong, _VP, _VP]),
    ("lbm_sg_phase_pressure", ctypes.c_int, [_VP, _VP, ctypes.c_longlong, ctypes.c_double, _VP, _VP, _VP]),
    ("lbm_sg_shift", ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_double, _VP]),
    ("lbm_destroy", None, [_VP]),
    ("lbm_strerror", ctypes.c_char_p, [ctypes.c_int]),
]


def load(path=LIB_PATH):
    """Load liblbm.so and declare its signatures (idempotent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LbmLibraryMissing(
            f"{path} not found: build it with `python -m paper_1812_00118_gb300.build` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code):
    return load().lbm_strerror(code).decode()


def _check(code, what):
    if code != OK:
        raise LbmError(code, what)


def lattice_info(lattice):
    lib = load()
    Q = ctypes.c_int()
    c = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    _check(lib.lbm_lattice_info(lattice, ctypes.byref(Q), c, w), "lbm_lattice_info")
    q = Q.value
    return np.array(c[: 3 * q]).reshape(q, 3), np.array(w[:q])


def make_params(M=0.1, W=4.0, sigma=0.01, rho_L=0.001, rho_H=1.0, nu_L=0.1 / 6, nu_H=0.1 / 6,
                g=(0.0, 0.0, 0.0), force_mode=0, eps=1e-10, hocorr=1, store=F32, P_ref=0.0, g_scale=0.0,
                C_dtheta=0.0):
    p = lbm_params()
    p.M, p.W, p.sigma, p.rho_L, p.rho_H, p.nu_L, p.nu_H = M, W, sigma, rho_L, rho_H, nu_L, nu_H
    for a in range(3):
        p.g[a] = g[a] if a < len(g) else 0.0
    p.force_mode, p.eps, p.hocorr, p.store = force_mode, eps, int(hocorr), store
    p.P_ref, p.g_scale = P_ref, g_scale
    p.C_dtheta = C_dtheta
    return p


def layout(lattice, shape, params, bc=(PERIODIC, PERIODIC, PERIODIC), ghost_band=False):
    """lbm_layout on the host (no GPU needed): dict of the padded extents px,
    py, pz of the population arrays (internal axes), cells per array, bytes of
    the population buffers and bytes of an initialised context."""
    g = lbm_grid()
    g.nx, g.ny = int(shape[0]), int(shape[1])
    g.nz = int(shape[2]) if lattice == D3Q19 else 1
    for a in range(3):
        g.bc[a] = bc[a] if a < len(bc) else PERIODIC
    out = (ctypes.c_longlong * 6)()
    _check(load().lbm_layout(ctypes.byref(g), lattice, ctypes.byref(params), CREATE_GHOST_BAND if ghost_band else 0,
                             out), "lbm_layout")
    return dict(px=out[0], py=out[1], pz=out[2], cells=out[3], population_bytes=out[4], context_bytes=out[5])


def _ptr(a, writable=False, n=None, device=None, name="field"):
    """(pointer, on_device) for a numpy float64 C-contiguous array or a contiguous
    torch float64 tensor (CUDA: device pointer; CPU, e.g. pinned: host pointer).
    n: the exact number of elements the library reads or writes; device: the
    CUDA device a device tensor must live on.  Either mismatch is a ValueError
    before anything reaches the library, which copies n elements unchecked."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: fields must be C-contiguous float64 arrays")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError(f"{name}: output array is read-only")
        if n is not None and a.size != n:
            raise ValueError(f"{name}: {n} elements required, got {a.size}")
        return ctypes.c_void_p(a.ctypes.data), 0
    if not hasattr(a, "data_ptr"):
        raise ValueError(f"{name}: a numpy array or a torch tensor is required, got {type(a).__name__}")
    if not (a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()):
        raise ValueError(f"{name}: tensor fields must be contiguous float64")
    if n is not None and a.numel() != n:
        raise ValueError(f"{name}: {n} elements required, got {a.numel()}")
    if a.is_cuda and device is not None and a.device.index != device:
        raise ValueError(f"{name}: on cuda:{a.device.index}, the domain lives on cuda:{device}")
    return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0


NOALLOC_MAX_NODES = 33554432


def _noalloc_arg(name, t, n_min, n_exact=None):
    """A contiguous float64 CUDA tensor on the current device with the stated
    number of elements, else ValueError (checked before anything is launched:
    a bad pointer or a short array would reach the kernel unchecked)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required, got {type(t).__name__}")
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: float64 required, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if n_exact is not None and t.numel() != n_exact:
        raise ValueError(f"{name}: {n_exact} elements required, got {t.numel()}")
    if t.numel() < n_min:
        raise ValueError(f"{name}: at least {n_min} elements required, got {t.numel()}")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, current device is cuda:{torch.cuda.current_device()}")
    return ctypes.c_void_p(t.data_ptr())


def field_sums_noalloc(phi, P, v, rho_L, rho_dif, out, stream=None):
    """lbm_field_sums_noalloc on device tensors: phi, P (n,), v a sequence of up
    to 3 component tensors of n elements (or None), out a float64 CUDA tensor
    of at least 4 elements; all contiguous float64 on the current device."""
    comps = list(v or [])
    if len(comps) > 3:
        raise ValueError("v: at most 3 components")
    p_phi = _noalloc_arg("phi", phi, 0)
    n = phi.numel()
    p_P = _noalloc_arg("P", P, 0, n)
    ptrs = [None if c is None else _noalloc_arg(f"v[{k}]", c, 0, n) for k, c in enumerate(comps)]
    ptrs += [None] * (3 - len(ptrs))
    p_out = _noalloc_arg("out", out, 4)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().lbm_field_sums_noalloc(p_phi, p_P, ptrs[0], ptrs[1], ptrs[2], int(n), float(rho_L),
                                         float(rho_dif), p_out, ctypes.c_void_p(stream)),
           "lbm_field_sums_noalloc")


class Simulation:
    """One LB domain on the current CUDA device (owns an lbm_ctx).

    shape is the user grid (nx, ny) for D2Q9 or (nx, ny, nz) for D3Q19;
    bc is a per-axis tuple of PERIODIC / WALL; ghost_band=True keeps ghost
    cells along the periodic axes too (lbm_create_ex with
    LBM_CREATE_GHOST_BAND), which the bulk-copy step tile needs."""

    def __init__(self, lattice, shape, params, bc=(PERIODIC, PERIODIC, PERIODIC), stream=None, ghost_band=False):
        lib = load()
        self.lattice = lattice
        self.dim = 2 if lattice == D2Q9 else 3
        nx, ny = shape[0], shape[1]
        nz = shape[2] if self.dim == 3 else 1
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        g = lbm_grid()
        g.nx, g.ny, g.nz = nx, ny, nz
        for a in range(3):
            g.bc[a] = bc[a] if a < len(bc) else PERIODIC
        self.params = params
        self.Q = 9 if lattice == D2Q9 else 19
        import torch
        self._device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = stream
        ctx = ctypes.c_void_p()
        _check(lib.lbm_create_ex(ctypes.byref(g), lattice, ctypes.byref(params), ctypes.c_void_p(stream),
                                 CREATE_GHOST_BAND if ghost_band else 0, ctypes.byref(ctx)), "lbm_create_ex")
        self._ctx = ctx

    # -- lifetime
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            load().lbm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C-ABI calls
    def init_fields(self, phi, u, P, nonequilibrium=False):
        """Populations from (phi, u, P); with nonequilibrium, g also carries
        the Chapman-Enskog non-equilibrium part (lbm_init_fields_ex)."""
        N, dev = self.N, self._device
        (pp, d0), (pu, d1), (pP, d2) = (_ptr(phi, n=N, device=dev, name="phi"),
                                        _ptr(u, n=self.dim * N, device=dev, name="u"),
                                        _ptr(P, n=N, device=dev, name="P"))
        if not (d0 == d1 == d2):
            raise ValueError("phi, u and P must all be host or all device")
        if nonequilibrium:
            _check(load().lbm_init_fields_ex(self._ctx, pp, pu, pP, d0, INIT_NONEQ), "lbm_init_fields_ex")
        else:
            _check(load().lbm_init_fields(self._ctx, pp, pu, pP, d0), "lbm_init_fields")

    def step(self, n=1):
        _check(load().lbm_step(self._ctx, int(n)), "lbm_step")

    def step_profiled(self, n):
        """n steps; returns the summed duration (ms) of the step-kernel launches."""
        ms = ctypes.c_double()
        _check(load().lbm_step_profiled(self._ctx, int(n), ctypes.byref(ms)), "lbm_step_profiled")
        return ms.value

    def macro(self, phi=None, P=None, rho_u=None):
        """Fill the given outputs (host arrays or device tensors); allocate host
        arrays when none is given and return (phi, P, rho_u)."""
        if phi is None and P is None and rho_u is None:
            phi = np.empty(self.N)
            P = np.empty(self.N)
            rho_u = np.empty(self.dim * self.N)
        ptrs, dev = [], None
        for a, n, name in ((phi, self.N, "phi"), (P, self.N, "P"), (rho_u, self.dim * self.N, "rho_u")):
            if a is None:
                ptrs.append(None)
                continue
            p, d = _ptr(a, writable=True, n=n, device=self._device, name=name)
            dev = d if dev is None else dev
            if d != dev:
                raise ValueError("outputs must all be host or all device")
            ptrs.append(p)
        _check(load().lbm_macro(self._ctx, *ptrs, dev or 0), "lbm_macro")
        return phi, P, rho_u

    def get_populations(self, h=None, g=None):
        """(h, g), Q*N doubles each; both given (host arrays or device tensors)
        or neither (host arrays are allocated)."""
        if (h is None) != (g is None):
            raise ValueError("give both h and g or neither")
        if h is None:
            h = np.empty(self.Q * self.N)
            g = np.empty(self.Q * self.N)
        n = self.Q * self.N
        (ph, d0), (pg, d1) = (_ptr(h, True, n=n, device=self._device, name="h"),
                              _ptr(g, True, n=n, device=self._device, name="g"))
        if d0 != d1:
            raise ValueError("h and g must both be host or both device")
        _check(load().lbm_get_populations(self._ctx, ph, pg, d0), "lbm_get_populations")
        return h, g

    def set_populations(self, h, g):
        n = self.Q * self.N
        (ph, d0), (pg, d1) = (_ptr(h, n=n, device=self._device, name="h"),
                              _ptr(g, n=n, device=self._device, name="g"))
        if d0 != d1:
            raise ValueError("h and g must both be host or both device")
        _check(load().lbm_set_populations(self._ctx, ph, pg, d0), "lbm_set_populations")

    def diagnostics(self, raise_on_divergence=True):
        out = (ctypes.c_double * 4)()
        rc = load().lbm_diagnostics(self._ctx, out)
        if rc not in (OK, EDIVERGED) or (rc == EDIVERGED and raise_on_divergence):
            _check(rc, "lbm_diagnostics")
        return dict(sum_phi=out[0], sum_rho=out[1], max_u=out[2], nonfinite=out[3], status=rc)

    def laplace(self, centre, r_in, r_out):
        c = (ctypes.c_double * 3)(*[float(v) for v in (list(centre) + [0.0] * 3)[:3]])
        dP = ctypes.c_double()
        _check(load().lbm_laplace(self._ctx, c, r_in, r_out, ctypes.byref(dP)), "lbm_laplace")
        return dP.value

    def launch_count(self):
        return load().lbm_launch_count(self._ctx)

    def set_phi_correction(self, every):
        """Re-impose the total of phi every `every` steps (0: never)."""
        _check(load().lbm_set_phi_correction(self._ctx, int(every)), "lbm_set_phi_correction")

    def set_wall_velocity(self, axis, side, u):
        """Velocity of the wall at end `side` (0 low, 1 high) of walled axis `axis`."""
        v = (ctypes.c_double * 3)(*[float(a) for a in (list(u) + [0.0, 0.0, 0.0])[:3]])
        _check(load().lbm_set_wall_velocity(self._ctx, int(axis), int(side), v), "lbm_set_wall_velocity")

    def set_tile(self, tile, lz):
        _check(load().lbm_set_tile(self._ctx, tile, lz), "lbm_set_tile")

    def set_wait_limit(self, polls):
        """Poll limit of the bulk-copy pipeline waits (0: give up at once)."""
        _check(load().lbm_set_wait_limit(self._ctx, int(polls)), "lbm_set_wait_limit")

    def get_tile(self):
        t, lz, tx, ty = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().lbm_get_tile(self._ctx, ctypes.byref(t), ctypes.byref(lz), ctypes.byref(tx),
                                   ctypes.byref(ty)), "lbm_get_tile")
        return t.value, lz.value, tx.value, ty.value

    def autotune(self, steps=20):
        """Pick the fastest tile/lz for this grid (state is restored); returns
        (tile, lz, ms_per_step)."""
        t, lz, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(load().lbm_autotune(self._ctx, int(steps), ctypes.byref(t), ctypes.byref(lz), ctypes.byref(ms)),
               "lbm_autotune")
        return t.value, lz.value, ms.value

    @property
    def ctx(self):
        return self._ctx


class _GridView(Simulation):
    """Grid i of a Batch: the per-grid calls of Simulation on the batch's
    view context (stepping it raises; the batch steps all grids)."""

    def __init__(self, batch, ctx, shape, params):
        self.lattice = D2Q9
        self.dim = 2
        self.shape = (shape[0], shape[1], 1)
        self.N = shape[0] * shape[1]
        self.Q = 9
        self.params = params
        self._stream = batch._stream
        self._device = batch._device
        self._ctx = ctx
        self._batch = batch   # keeps the batch (owner of the context) alive

    def close(self):
        self._ctx = None


def _grids(shapes, bcs):
    arr = (lbm_grid * len(shapes))()
    for i, sh in enumerate(shapes):
        arr[i].nx, arr[i].ny, arr[i].nz = int(sh[0]), int(sh[1]), 1
        bc = bcs[i] if bcs is not None else (PERIODIC, PERIODIC)
        for a in range(3):
            arr[i].bc[a] = bc[a] if a < len(bc) else PERIODIC
    return arr


def plan(shapes, tx, lz):
    """Work list of a batch of D2Q9 grids (host computation): (m, 4) int array of
    (grid, x0, z0, z1) with internal z = user y."""
    lib = load()
    g = _grids(shapes, None)
    m = lib.lbm_batch_plan(len(shapes), g, int(tx), int(lz), None, 0)
    if m < 0:
        _check(m, "lbm_batch_plan")
    out = (ctypes.c_int * (4 * max(m, 1)))()
    _check(min(0, lib.lbm_batch_plan(len(shapes), g, int(tx), int(lz), out, m)), "lbm_batch_plan")
    return np.array(out[: 4 * m], dtype=np.int64).reshape(m, 4)


class Batch:
    """Many D2Q9 grids in one set of population arrays, stepped by one
    persistent launch per step (owns an lbm_batch).

    shapes: sequence of (nx, ny); params: one lbm_params for all grids or a
    sequence (same storage type); bcs: optional per-grid (bc_x, bc_y)."""

    def __init__(self, shapes, params, bcs=None, stream=None):
        lib = load()
        n = len(shapes)
        plist = list(params) if isinstance(params, (list, tuple)) else [params] * n
        if len(plist) != n:
            raise ValueError("one parameter block per grid")
        parr = (lbm_params * n)(*plist)
        import torch
        self._device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = stream
        self.shapes = [(int(a), int(b)) for a, b in shapes]
        self.params = plist
        b = ctypes.c_void_p()
        _check(lib.lbm_batch_create(n, _grids(shapes, bcs), parr, ctypes.c_void_p(stream), ctypes.byref(b)),
               "lbm_batch_create")
        self._b = b
        self._views = [None] * n

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            for v in self._views:
                if v is not None:
                    v.close()
            load().lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.shapes)

    def grid(self, i):
        if self._views[i] is None:
            ctx = load().lbm_batch_grid(self._b, int(i))
            if not ctx:
                raise IndexError(i)
            self._views[i] = _GridView(self, ctypes.c_void_p(ctx), self.shapes[i], self.params[i])
        return self._views[i]

    def step(self, n=1):
        _check(load().lbm_batch_step(self._b, int(n)), "lbm_batch_step")

    def step_sequential(self, n=1):
        _check(load().lbm_batch_step_sequential(self._b, int(n)), "lbm_batch_step_sequential")

    def set_tile(self, tile, lz):
        _check(load().lbm_batch_set_tile(self._b, int(tile), int(lz)), "lbm_batch_set_tile")

    def get_tile(self):
        t, lz, tx, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().lbm_batch_get_tile(self._b, ctypes.byref(t), ctypes.byref(lz), ctypes.byref(tx),
                                         ctypes.byref(m)), "lbm_batch_get_tile")
        return t.value, lz.value, tx.value, m.value

    def set_graph(self, k):
        _check(load().lbm_batch_set_graph(self._b, int(k)), "lbm_batch_set_graph")

    def autotune(self, steps=10):
        t, lz, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(load().lbm_batch_autotune(self._b, int(steps), ctypes.byref(t), ctypes.byref(lz), ctypes.byref(ms)),
               "lbm_batch_autotune")
        return t.value, lz.value, ms.value

    def launch_count(self):
        return load().lbm_batch_launch_count(self._b)
