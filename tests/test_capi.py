"""Host-side checks of the C-ABI (no GPU needed): the library builds, loads,
exports every function include/*.h declares, and reports a velocity set
equal to the oracle's up to ordering."""
import os
import re

import numpy as np
import pytest

from oracle import lattice as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_00118_gb300 import build, lbm
    build.build()
    return lbm.load()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm\w*)\s*\(", text))
    return sorted(names)


def test_header_symbols_exported(lib):
    from paper_1812_00118_gb300 import lbm
    names = declared_functions()
    assert len(names) >= 14
    bound = {n for n, _, _ in lbm.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"
        assert n in bound, f"{n} has no Python binding"


@pytest.mark.parametrize("lat_id,olat", [(0, L.D2Q9), (1, L.D3Q19)], ids=["D2Q9", "D3Q19"])
def test_lattice_info_matches_oracle(lib, lat_id, olat):
    from paper_1812_00118_gb300 import lbm
    c, w = lbm.lattice_info(lat_id)
    assert len(w) == olat.Q
    ours = {tuple(v): wv for v, wv in zip(c.tolist(), w)}
    theirs = {tuple(int(a) for a in v): wv for v, wv in zip(olat.c, olat.w)}
    assert ours.keys() == theirs.keys()
    for k in ours:
        assert ours[k] == pytest.approx(theirs[k], abs=1e-16)


def test_strerror(lib):
    from paper_1812_00118_gb300 import lbm
    assert lbm.strerror(0) == "ok"
    assert "invalid" in lbm.strerror(-1)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1812_00118_gb300 import lbm
    saved = lbm._lib
    lbm._lib = None
    try:
        with pytest.raises(lbm.LbmLibraryMissing):
            lbm.load(str(tmp_path / "nope.so"))
    finally:
        lbm._lib = saved


def test_noalloc_binding_rejects_bad_arguments_before_launch():
    """The binding of lbm_field_sums_noalloc checks every argument before it
    reaches the library: a numpy array, a wrong dtype, a non-contiguous
    tensor, a P or vector component shorter than phi, an output of fewer than
    4 elements, or a tensor not on the current CUDA device is a ValueError
    (on this CPU-only machine every tensor fails the device check last)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_1812_00118_gb300 import lbm
    f = torch.zeros(10, dtype=torch.float64)
    out = torch.zeros(4, dtype=torch.float64)
    bad = [
        (np.zeros(10), f, None, out),                               # not a tensor
        (f.float(), f, None, out),                                  # dtype
        (torch.zeros(10, 2, dtype=torch.float64)[:, 0], f, None, out),   # not contiguous
        (f, torch.zeros(9, dtype=torch.float64), None, out),        # P shorter than phi
        (f, f, [f, torch.zeros(3, dtype=torch.float64)], out),      # component shorter
        (f, f, [f, f, f, f], out),                                  # four components
        (f, f, None, torch.zeros(3, dtype=torch.float64)),          # out too short
        (f, f, None, out),                                          # host tensors
    ]
    for phi, P, v, o in bad:
        with pytest.raises(ValueError):
            lbm.field_sums_noalloc(phi, P, v, 0.0, 1.0, o, stream=0)


def test_create_rejects_bad_arguments_before_any_allocation(lib):
    """lbm_create_ex validates its grid, parameters and flags before it touches
    the GPU: an unknown flag, a D2Q9 grid with nz != 1, a bad boundary type or
    a non-positive mobility return LBM_EINVAL and no context (this machine has
    no GPU, so reaching an allocation would fail differently)."""
    import ctypes
    from paper_1812_00118_gb300 import lbm
    prm = lbm.make_params()
    ctx = ctypes.c_void_p()

    def create(grid, lattice=lbm.D3Q19, params=prm, flags=0):
        ctx.value = None
        rc = lib.lbm_create_ex(ctypes.byref(grid), lattice, ctypes.byref(params), None, flags, ctypes.byref(ctx))
        return rc, ctx.value

    g = lbm.lbm_grid()
    g.nx, g.ny, g.nz = 16, 16, 16
    assert create(g, flags=2) == (lbm.EINVAL, None)                       # unknown flag
    assert create(g, flags=lbm.CREATE_GHOST_BAND | 4) == (lbm.EINVAL, None)
    g2 = lbm.lbm_grid()
    g2.nx, g2.ny, g2.nz = 16, 16, 2
    assert create(g2, lattice=lbm.D2Q9) == (lbm.EINVAL, None)            # D2Q9 with nz != 1
    g3 = lbm.lbm_grid()
    g3.nx, g3.ny, g3.nz = 16, 16, 16
    g3.bc[1] = 7
    assert create(g3) == (lbm.EINVAL, None)                              # unknown boundary type
    bad = lbm.make_params(M=0.0)
    assert create(g, params=bad) == (lbm.EINVAL, None)                   # M must be positive
    inf, nan = float("inf"), float("nan")
    for kw in (dict(nu_L=inf), dict(rho_H=inf), dict(sigma=nan), dict(g=(nan, 0.0, 0.0)), dict(eps=inf),
               dict(store=lbm.F16S, P_ref=nan), dict(store=lbm.F16S, g_scale=-1.0), dict(C_dtheta=inf)):
        assert create(g, params=lbm.make_params(**kw)) == (lbm.EINVAL, None), kw   # not finite / negative scale


def test_simulation_binding_rejects_wrong_sizes_before_any_call(lib):
    """Simulation.init_fields / macro / get_populations / set_populations
    check the element count of every field before the library copies it: phi
    and P must hold N doubles, u and rho u dim*N, h and g Q*N (a short device
    tensor would otherwise be read or written past its end on the GPU).  The
    object is made without a context, so a check that let a bad field through
    would reach the library with a NULL context and fail differently."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_1812_00118_gb300 import lbm
    sim = lbm.Simulation.__new__(lbm.Simulation)
    sim.lattice, sim.dim, sim.Q = lbm.D2Q9, 2, 9
    sim.shape, sim.N, sim._device, sim._ctx = (6, 5, 1), 30, 0, None
    N = sim.N
    z = np.zeros
    bad_init = [
        (z(N - 1), z(2 * N), z(N)),          # phi short
        (z(N), z(3 * N), z(N)),              # u with 3 components on D2Q9
        (z(N), z(2 * N), z(N + 1)),          # P long
        (z(N).astype(np.float32), z(2 * N), z(N)),                      # dtype
        (z((N, 2))[:, 0], z(2 * N), z(N)),                              # not contiguous
        (torch.zeros(N, dtype=torch.float64), torch.zeros(2 * N - 2, dtype=torch.float64),
         torch.zeros(N, dtype=torch.float64)),                          # tensor u short
        ([0.0] * N, z(2 * N), z(N)),                                    # not an array
    ]
    for phi, u, P in bad_init:
        with pytest.raises(ValueError):
            sim.init_fields(phi, u, P)
    with pytest.raises(ValueError):
        sim.macro(z(N), z(N), z(3 * N))
    with pytest.raises(ValueError):
        sim.macro(None, z(N - 1), None)
    ro = z(N)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        sim.macro(ro, None, None)
    with pytest.raises(ValueError):
        sim.get_populations(z(9 * N), None)              # one of the two
    with pytest.raises(ValueError):
        sim.get_populations(z(9 * N), z(9 * N - 1))
    with pytest.raises(ValueError):
        sim.set_populations(z(9 * N + 9), z(9 * N))
    # correctly sized fields pass the checks and reach the library, which
    # refuses the missing context
    for call in (lambda: sim.init_fields(z(N), z(2 * N), z(N)),
                 lambda: sim.macro(z(N), z(N), z(2 * N)),
                 lambda: sim.get_populations(z(9 * N), z(9 * N)),
                 lambda: sim.set_populations(z(9 * N), z(9 * N))):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.code == lbm.EINVAL


def test_surrogate_binding_rejects_bad_targets_before_any_call(lib):
    """Surrogate.backward hands the target pointer to the loss kernel, which
    reads M x 4 floats: anything but a contiguous float32 CUDA tensor of that
    shape on the network's device is a ValueError first (on this CPU-only
    machine every tensor also fails the device test), and set_input refuses
    a wrong shape."""
    torch = pytest.importorskip("torch")
    from paper_1812_00118_gb300 import surrogate as SG
    sg = SG.Surrogate.__new__(SG.Surrogate)
    sg.torch, sg.lib, sg.stream, sg.a, sg.M = torch, lib, 0, {}, [64, 16, 4, 1]
    sg.x32 = torch.zeros(64, 4)
    for t in (torch.zeros(64, 4, dtype=torch.float64), torch.zeros(63, 4), torch.zeros(4, 64).t(),
              torch.zeros(64, 4)):
        with pytest.raises(ValueError):
            sg.backward(t)
    with pytest.raises(ValueError):
        sg.set_input(torch.zeros(32, 4))


def test_create_rejects_grids_whose_padded_size_overflows(lib):
    """A grid whose padded size reaches 2^31 cells is refused before any
    allocation, including sizes whose x-y plane alone overflows 32 bits
    (65536 x 65536 x 1 would wrap to an empty plane in 32-bit arithmetic)."""
    import ctypes
    from paper_1812_00118_gb300 import lbm
    prm = lbm.make_params()
    ctx = ctypes.c_void_p()
    for nx, ny, nz in ((65536, 65536, 1), (65536, 65536, 2), (2048, 1024, 1024), (1 << 30, 4, 1),
                       (2147483647, 1, 1)):
        g = lbm.lbm_grid()
        g.nx, g.ny, g.nz = nx, ny, nz
        ctx.value = None
        rc = lib.lbm_create_ex(ctypes.byref(g), lbm.D3Q19, ctypes.byref(prm), None, 0, ctypes.byref(ctx))
        assert (rc, ctx.value) == (lbm.EINVAL, None), (nx, ny, nz)
    # a D2Q9 grid of 65536 x 32768 (2^31 cells) too
    g = lbm.lbm_grid()
    g.nx, g.ny, g.nz = 65536, 32768, 1
    rc = lib.lbm_create_ex(ctypes.byref(g), lbm.D2Q9, ctypes.byref(prm), None, 0, ctypes.byref(ctx))
    assert rc == lbm.EINVAL


@pytest.mark.parametrize("store,elem", [(0, 8), (1, 4), (2, 2), (3, 2)], ids=["f64", "f32", "f16s", "bf16s"])
def test_layout_plan_on_the_host(lib, store, elem):
    """lbm_layout reports the padded layout of the population arrays without
    a GPU: x rows padded to 32 bytes; ghost cells only along walled axes
    (32 bytes of x, at least 2 cells; 2 in y; one plane in z), or along every
    axis with the ghost band; population buffers of 4 Q cells x the element
    size (h and g at two time levels); the context's total adds the 5 N
    doubles of scratch fields and the reduction partials."""
    from paper_1812_00118_gb300 import lbm
    prm = lbm.make_params(store=store)
    a32 = 32 // elem
    gx = max(a32, 2)
    pad = lambda n: (n + a32 - 1) // a32 * a32
    for shape, bc, band in (((128, 128, 128), (0, 0, 0), False), ((37, 21, 13), (1, 0, 1), False),
                            ((37, 21, 13), (0, 1, 0), False), ((37, 21, 13), (0, 0, 0), True)):
        L_ = lbm.layout(lbm.D3Q19, shape, prm, bc=bc, ghost_band=band)
        nx, ny, nz = shape
        wx, wy, wz = (band or bc[0] == 1), (band or bc[1] == 1), (band or bc[2] == 1)
        assert L_["px"] == pad(nx) + (2 * gx if wx else 0)
        assert L_["py"] == ny + (4 if wy else 0)
        assert L_["pz"] == nz + (2 if wz else 0)
        assert L_["px"] * elem % 32 == 0
        assert L_["cells"] == L_["px"] * L_["py"] * L_["pz"]
        assert L_["population_bytes"] == 4 * 19 * L_["cells"] * elem
        assert L_["context_bytes"] == L_["population_bytes"] + 4 + 40 * nx * ny * nz + 8 * 8 * 1024
    # D2Q9: the user's y is the internal z; no y ghosts
    L2 = lbm.layout(lbm.D2Q9, (100, 60), prm, bc=(1, 1))
    assert (L2["px"], L2["py"], L2["pz"]) == (pad(100) + 2 * gx, 1, 62)
    assert L2["population_bytes"] == 4 * 9 * L2["cells"] * elem


def test_layout_refuses_what_create_refuses(lib):
    from paper_1812_00118_gb300 import lbm
    prm = lbm.make_params()
    for lattice, shape in ((lbm.D3Q19, (65536, 65536, 1)), (lbm.D3Q19, (0, 8, 8)), (lbm.D2Q9, (65536, 32768))):
        with pytest.raises(lbm.LbmError) as e:
            lbm.layout(lattice, shape, prm)
        assert e.value.code == lbm.EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.layout(lbm.D3Q19, (8, 8, 8), lbm.make_params(M=0.0))
    # the largest FP32 cube within the 2^31-cell limit of one population array
    ok = lbm.layout(lbm.D3Q19, (1288, 1288, 1288), prm)
    assert ok["cells"] < 2 ** 31
    with pytest.raises(lbm.LbmError):
        lbm.layout(lbm.D3Q19, (1296, 1296, 1296), prm)


def test_surrogate_calls_validate_arguments_on_the_host(lib):
    """The surrogate kernels' C-ABI refuses bad arguments before any device
    call: NULL operands, channel counts that are not multiples of 16 or above
    128 outputs, operands off their 16-byte boundary, strides below the
    channel count, pooling factors that do not divide the grid, negative
    pixel counts, an Adam step below 1, an unstable diffusion coefficient and
    a bulk-phase threshold of 1/2 or more all return LBM_EINVAL.  The
    addresses passed are never dereferenced (this machine has no GPU)."""
    import ctypes
    from paper_1812_00118_gb300 import lbm
    V = ctypes.c_void_p
    p = V(1 << 14)                      # 16-byte aligned, not NULL
    cases = [
        lambda: lib.lbm_sg_conv3x3(None, 16, p, None, p, 16, 1, 8, 128, 16, 16, None),
        lambda: lib.lbm_sg_conv3x3(p, 16, p, None, p, 16, 1, 8, 128, 8, 16, None),
        lambda: lib.lbm_sg_conv3x3(p, 144, p, None, p, 144, 1, 8, 128, 16, 144, None),
        lambda: lib.lbm_sg_conv3x3(V((1 << 14) + 2), 16, p, None, p, 16, 1, 8, 128, 16, 16, None),
        lambda: lib.lbm_sg_conv3x3(p, 8, p, None, p, 16, 1, 8, 128, 16, 16, None),
        lambda: lib.lbm_sg_pool(p, 16, p, 16, 1, 8, 8, 16, 3, None),
        lambda: lib.lbm_sg_relu(p, 16, p, 16, -1, 16, None),
        lambda: lib.lbm_sg_adam(p, p, p, p, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None, None),
        lambda: lib.lbm_sg_smooth(p, p, 1, 8, 8, 1, 0.3, None),
        lambda: lib.lbm_sg_phase_pressure(p, p, 10, 0.6, p, p, None),
    ]
    for k, call in enumerate(cases):
        assert call() == lbm.EINVAL, k


def test_every_entry_point_is_documented():
    """Every function include/*.h declares is preceded by its comment block
    (what it computes, the arguments' meaning and layout, ownership, errors)
    or belongs to the group a block describes."""
    decl = re.compile(r"^(?:int|void|long long|const char\*|lbm_ctx\*|void\*)\s+\*?(lbm\w+)\s*\(")
    undocumented = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", f)).read().split("\n")
        for i, line in enumerate(lines):
            m = decl.match(line)
            if not m:
                continue
            j = i - 1
            while j >= 0 and (not lines[j].strip() or decl.match(lines[j])
                              or (lines[j].startswith(" ") and not lines[j].strip().startswith("*"))):
                j -= 1
            prev = lines[j].strip() if j >= 0 else ""
            if not (prev.endswith("*/") or prev.startswith("#define")):
                undocumented.append(f"{f}: {m.group(1)}")
    assert not undocumented, undocumented
