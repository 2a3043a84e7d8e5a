"""Learned warm start of the phase-field LB solver, and time-to-tolerance.

A state of drops and bubbles relaxes slowly from its initial fields:
starting from u = 0, P = 0 the Laplace pressure jumps build up as acoustic
waves that the viscosity damps over tens of thousands of steps.  The
surrogate (paper_1812_00118_gb300.surrogate, a four-level U-Net) learns the
map of the state (phi, rho u, P) over DT = 2000 steps from snapshot pairs
the solver itself generates (1-4 drops or bubbles, radii 12-48, density
ratio 1000).  At inference it is applied k times to the initial fields,
jumping k DT steps ahead towards the end of the transient; the populations
are rebuilt from the prediction as equilibria plus the filtered
non-equilibrium part (lbm_init_fields_ex, LBM_INIT_NONEQ), after the
predicted phi is projected onto the start (change confined to the
interfaces, total of phi restored in FP64: lbm_sg_phi_project).  The plain
solver then continues and decides convergence: the network only chooses
the state the solver starts from, so a poor prediction costs steps, not
accuracy.

Convergence (time-to-tolerance): every `check_every` steps the Laplace
jump of the state, J = mean P of the bulk heavy phase minus mean P of the
bulk light phase, is compared with its value `check_every` steps before;
the run has converged when |J(t) - J(t - k)| / |J(t)| < tol for
`consecutive` checks in a row (FP64 sums on the GPU,
lbm_sg_phase_pressure).  The node-wise pressure residual ||P(t) - P(t - k)||
/ ||P(t)|| is available too; FP32 rounding noise keeps it above ~1e-5.

Everything that computes runs in the library's kernels; PyTorch allocates
device memory and copies it.
"""
import ctypes

import numpy as np

from . import inputs as I
from . import lbm as L
from .surrogate import NC, _ck, _ptr

# normalisation of (phi, rho u_x, rho u_y, P) for the network: over the
# transient both rho u and P have a standard deviation of ~2e-4 - 3e-4
# (the Laplace jumps sigma / R are 2e-4 - 1e-3), so every channel of the
# network's input is O(1)
SCALE = (1.0, 2e-4, 2e-4, 3e-4)
# the warm-start workload: drops and bubbles at density ratio 1000, the
# water-like viscosity of the paper's shear and Galilean tests
PHYS = dict(M=0.1, W=4.0, sigma=0.01, rho_L=1e-3, rho_H=1.0, nu_L=1.0 / 60.0, nu_H=1.0 / 60.0)
RADII = (12.0, 48.0)
DT = 2000          # steps between the snapshots of a training pair


def case_params(store=L.F32):
    return L.make_params(store=store, g_scale=(1e3 if store == L.F16S else 0.0), **PHYS)


def case_fields(Lsz, seed, R_min=RADII[0], R_max=RADII[1], bubbles=None):
    """phi (flat) of case `seed`: 1-4 drops, or (odd seeds) 1-4 bubbles,
    three interface widths apart (static, no coalescence); and their
    (x, y, R)."""
    b = (seed % 2 == 1) if bubbles is None else bubbles
    R_max = min(R_max, Lsz / 4.0)
    phi, u, P, placed = I.drops(Lsz, seed, R_min=R_min, R_max=R_max, W=PHYS["W"], gap=3.0 * PHYS["W"], bubbles=b)
    return phi.reshape(-1).copy(), placed


class DeviceFields:
    """FP64 device fields of one grid (phi, P, rho u as lbm_macro writes them,
    and u for lbm_init_fields)."""

    def __init__(self, torch, n):
        z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
        self.n = n
        self.phi, self.P, self.ru, self.u = z(n), z(n), z(2 * n), z(2 * n)


def _scale_arr():
    return (ctypes.c_double * 4)(*SCALE)


def pack(lib, f, x32, x16, stream):
    """x32/x16 (device addresses) <- (phi, rho u, P) of f."""
    n = f.n
    ru = f.ru.data_ptr()
    _ck(lib.lbm_sg_pack(_ptr(f.phi), ctypes.c_void_p(ru), ctypes.c_void_p(ru + 8 * n), _ptr(f.P), _scale_arr(),
                        ctypes.c_void_p(x32), NC, ctypes.c_void_p(x16), 16, n, stream), "lbm_sg_pack")


def generate_snapshots(torch, Lsz, seeds, K, dt=DT, store=L.F32, max_u=0.05, chunk=256):
    """Trajectories of the batched solver: for every case the normalised
    state at t = 0, dt, ..., K dt as an (n, K + 1, L*L, 4) float32 device
    tensor; cases whose run does not stay bounded (non-finite fields or
    |u| > max_u at some snapshot) are left out.  Returns (S, n_left_out).
    Cases run `chunk` at a time as one batch."""
    lib = L.load()
    npix = Lsz * Lsz
    prm = case_params(store)
    stream = torch.cuda.current_stream().cuda_stream
    tmp16 = torch.zeros(npix, 16, dtype=torch.bfloat16, device="cuda")
    f = DeviceFields(torch, npix)
    kept = []
    dropped = 0
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0:c0 + chunk]
        n = len(part)
        S = torch.zeros(n, K + 1, npix, NC, dtype=torch.float32, device="cuda")
        batch = L.Batch([(Lsz, Lsz)] * n, prm, stream=stream)
        for k, sd in enumerate(part):
            phi0, _ = case_fields(Lsz, sd)
            f.phi.copy_(torch.from_numpy(phi0))
            for t in (f.P, f.ru, f.u):
                t.zero_()
            batch.grid(k).init_fields(f.phi, f.u, f.P)
        ok = [True] * n

        def record(j):
            for k in range(n):
                if not ok[k]:
                    continue
                d = batch.grid(k).diagnostics(raise_on_divergence=False)
                if d["nonfinite"] > 0 or not d["max_u"] < max_u:
                    ok[k] = False
                    continue
                batch.grid(k).macro(f.phi, f.P, f.ru)
                pack(lib, f, S[k, j].data_ptr(), tmp16.data_ptr(), stream)

        record(0)
        for j in range(1, K + 1):
            batch.step(dt)
            record(j)
        torch.cuda.synchronize()
        batch.close()
        idx = [k for k in range(n) if ok[k]]
        dropped += n - len(idx)
        if idx:
            kept.append(S.index_select(0, torch.tensor(idx, dtype=torch.long, device="cuda")))
        del S
    if not kept:
        raise RuntimeError(f"generate_snapshots: all {dropped} cases left the bounds (non-finite or |u| >= {max_u})")
    return torch.cat(kept, 0), dropped


def train(torch, sg, S, iters, lr=1e-3, seed=0, log_every=100, decay_at=0.7):
    """Adam on random mini-batches of sg.N pairs (snapshot k of a case as
    input, snapshot k + 1 as target; indices drawn on the host); the learning
    rate drops tenfold after decay_at of the iterations.  Returns
    [(iteration, loss)]."""
    rng = np.random.default_rng(seed)
    n, K1, npix = S.shape[0], S.shape[1], S.shape[2]
    xb = torch.zeros(sg.N * npix, NC, dtype=torch.float32, device="cuda")
    yb = torch.zeros_like(xb)
    hist = []
    for it in range(iters):
        cs = rng.integers(0, n, size=sg.N)
        ks = rng.integers(0, K1 - 1, size=sg.N)
        for j, (c, k) in enumerate(zip(cs, ks)):   # gather the mini-batch (device copies)
            xb[j * npix:(j + 1) * npix].copy_(S[int(c), int(k)])
            yb[j * npix:(j + 1) * npix].copy_(S[int(c), int(k) + 1])
        loss = sg.train_step(xb, yb, lr=lr if it < decay_at * iters else 0.1 * lr)
        if it % log_every == 0 or it == iters - 1:
            hist.append((it, float(loss.item())))
    return hist


def identity_loss(S):
    """MSE of the map that keeps the state (the loss to beat)."""
    return float(((S[:, 1:] - S[:, :-1]) ** 2).mean().item())


def predict_into(torch, sg1, sim, phi0_host, prm, k_apply, velocity=True):
    """Warm start: apply the one-image surrogate k_apply times to the initial
    fields (phi0, 0, 0) -- a jump of k_apply DT steps --, project the
    predicted phi onto the start (its change kept to the start's interface
    band, clipped to [0, 1], the total of phi0 restored by moving the
    interfaces: lbm_sg_phi_project), and rebuild sim's populations from
    (phi, u, P) as equilibria plus the Chapman-Enskog non-equilibrium part.
    u = (predicted rho u) / rho(projected phi), or 0 without `velocity`.
    Returns the fields."""
    lib = L.load()
    n = sg1.M[0]
    stream = torch.cuda.current_stream().cuda_stream
    f = DeviceFields(torch, n)
    phi0 = torch.from_numpy(phi0_host).cuda()
    f.phi.copy_(phi0)
    tmp16 = torch.zeros(n, 16, dtype=torch.bfloat16, device="cuda")
    x32 = torch.zeros(n, NC, dtype=torch.float32, device="cuda")
    x32n = torch.zeros_like(x32)
    pack(lib, f, x32.data_ptr(), tmp16.data_ptr(), stream)
    delta = None
    for k in range(k_apply):
        if delta is not None:   # x <- x + delta of the previous application
            _ck(lib.lbm_sg_add(_ptr(x32), NC, _ptr(delta), 16, _ptr(x32n), NC, n, NC, stream), "lbm_sg_add")
            x32, x32n = x32n, x32
        sg1.set_input(x32)
        delta = sg1.forward()
    u = f.u.data_ptr()
    rho_dif = prm.rho_H - prm.rho_L
    if delta is None:
        delta = torch.zeros(n, 16, dtype=torch.float32, device="cuda")
    unpack = lambda phi_out, phi_rho: _ck(lib.lbm_sg_unpack(
        _ptr(x32), NC, _ptr(delta), 16, _ptr(phi_out), ctypes.c_void_p(u), ctypes.c_void_p(u + 8 * n), _ptr(f.P),
        _scale_arr(), prm.rho_L, rho_dif, phi_rho, n, stream), "lbm_sg_unpack")
    unpack(f.phi, None)
    scratch = torch.zeros(769, dtype=torch.float64, device="cuda")
    _ck(lib.lbm_sg_phi_project(_ptr(f.phi), _ptr(phi0), n, _ptr(scratch), stream), "lbm_sg_phi_project")
    if velocity:   # u again, now over the density of the projected phi
        unpack(torch.empty_like(f.phi), _ptr(f.phi))
    else:
        f.u.zero_()
    sim.init_fields(f.phi, f.u, f.P, nonequilibrium=True)
    return f


class _Residual:
    """The convergence measure of one grid, on the GPU in FP64.

    "laplace" (default): J = mean P of the bulk heavy phase (phi >= 0.99)
    minus mean P of the bulk light phase (phi <= 0.01), the Laplace jump of
    the whole state (lbm_sg_phase_pressure); r = |J(t) - J(t - k)| / |J(t)|.
    "field": r = ||P(t) - P(t - k)|| / ||P(t)|| over every node
    (lbm_sg_residual), which FP32 rounding noise of the pressure field keeps
    above ~1e-5."""

    def __init__(self, torch, sim, measure="laplace"):
        self.lib, self.sim, self.measure = L.load(), sim, measure
        self.stream = torch.cuda.current_stream().cuda_stream
        n = sim.N
        z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
        self.phi, self.P = z(n), [z(n), z(n)]
        self.out, self.scratch = z(4), z(1024)
        self.cur, self.J = 0, None
        self._read()

    def _read(self):
        self.sim.macro(self.phi, self.P[self.cur], None)
        if self.measure == "laplace":
            _ck(self.lib.lbm_sg_phase_pressure(_ptr(self.phi), _ptr(self.P[self.cur]), self.sim.N, 0.01,
                                               _ptr(self.out), _ptr(self.scratch), self.stream),
                "lbm_sg_phase_pressure")
            o = self.out.tolist()
            self.J = o[0] - o[1]

    def update(self):
        """Read the fields again; the residual against the previous read."""
        prev_J = self.J
        self.cur = 1 - self.cur
        self._read()
        if self.measure == "laplace":
            return abs(self.J - prev_J) / abs(self.J) if self.J != 0 else float("inf")
        _ck(self.lib.lbm_sg_residual(_ptr(self.P[self.cur]), _ptr(self.P[1 - self.cur]), self.sim.N, _ptr(self.out),
                                     _ptr(self.scratch), self.stream), "lbm_sg_residual")
        d2, a2 = self.out.tolist()[:2]
        return float(np.sqrt(d2 / a2)) if a2 > 0 else float("inf")


def steps_to_tolerance(torch, sim, tol=1e-6, check_every=100, consecutive=3, max_steps=200000, measure="laplace",
                       history=None):
    """Steps until the residual (see _Residual) stays below tol for
    `consecutive` checks `check_every` steps apart (None if not within
    max_steps or if the run diverges); returns (steps, device ms of the
    whole loop including the checks, last residual).  `history`, a list,
    receives every residual."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = _Residual(torch, sim, measure)
    steps, ok, r, done = 0, 0, float("inf"), None
    while steps < max_steps:
        sim.step(check_every)
        steps += check_every
        r = res.update()
        if history is not None:
            history.append(r)
        if not np.isfinite(r):   # the run diverged: no convergence
            break
        ok = ok + 1 if r < tol else 0
        if ok >= consecutive:
            done = steps
            break
    e1.record()
    e1.synchronize()
    return done, e0.elapsed_time(e1), r


def batch_steps_to_tolerance(torch, batch, tol=1e-6, check_every=100, consecutive=3, max_steps=200000,
                             measure="laplace", on_converged=None):
    """steps_to_tolerance for every grid of a Batch stepped together: the
    batch advances until each grid has met the criterion (or max_steps);
    returns (per-grid steps or None, device ms of the whole loop).
    on_converged(k), if given, is called when grid k meets the criterion
    (the batch keeps stepping the grids that already have)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = [_Residual(torch, batch.grid(k), measure) for k in range(len(batch))]
    done = [None] * len(res)
    ok = [0] * len(res)
    steps = 0
    while steps < max_steps and any(d is None for d in done):
        batch.step(check_every)
        steps += check_every
        for k, rk in enumerate(res):
            if done[k] is not None:
                continue
            r = rk.update()
            ok[k] = ok[k] + 1 if r < tol else 0
            if ok[k] >= consecutive:
                done[k] = steps
                if on_converged is not None:
                    on_converged(k)
    e1.record()
    e1.synchronize()
    return done, e0.elapsed_time(e1)


def steps_at(history, tol, check_every=100, consecutive=3):
    """From a residual history: the steps at which the residual had first
    stayed below tol for `consecutive` checks (None if never)."""
    run = 0
    for i, r in enumerate(history):
        run = run + 1 if r < tol else 0
        if run >= consecutive:
            return (i + 1) * check_every
    return None


def laplace_error(sim, placed, bubble):
    """For a state of one drop (or one bubble, `bubble`): the Laplace jump
    (Section 4.1) across its interface against sigma / R, minus 1, measured
    around the current centre of the enclosed phase (circular mean over the
    periodic box, so a drop that has drifted is still found) with R from its
    area (2-D); None for several drops."""
    if len(placed) != 1:
        return None
    nx, ny, _ = sim.shape
    f, _, _ = sim.macro()
    if not np.isfinite(f).all():
        return None
    w = (1.0 - f if bubble else f).reshape(ny, nx).clip(0.0, 1.0)
    centre = []
    for prof, n in ((w.sum(axis=0), nx), (w.sum(axis=1), ny)):
        a = 2.0 * np.pi * np.arange(n) / n
        centre.append((np.arctan2((prof * np.sin(a)).sum(), (prof * np.cos(a)).sum()) % (2.0 * np.pi)) * n / (2.0 * np.pi))
    R = float(np.sqrt(w.sum() / np.pi))
    W = PHYS["W"]
    return sim.laplace(tuple(centre), R - 2.0 * W, R + 2.0 * W) / (PHYS["sigma"] / R) - 1.0
