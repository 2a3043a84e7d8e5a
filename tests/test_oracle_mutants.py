"""The oracle's pins against planted mistakes.

Each case plants one plausible slip -- a dropped term, a wrong sign, factor,
index or operand -- in a fresh copy of an oracle module (the LB step, or the
surrogate network's forward and backward pass), built in
this process from its source with one expression replaced (nothing on disk
changes), points the pin test's module at the copy, and requires the pin to
fail.  The pins named here check the oracle against what the paper and the
mathematics fix (moment identities, closed forms, stencil symbols,
conservation, relaxation rates, force balances), not against a second
transcription of the same formulas, so a slip they let through would leave
part of the oracle trusted on its own word.
"""
import importlib
import os
import sys
import types

import pytest

from oracle import lattice as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "oracle", "pflbm.py")).read()
SRC_SG = open(os.path.join(ROOT, "oracle", "surrogate.py")).read()
SRC_DG = open(os.path.join(ROOT, "oracle", "diagnostics.py")).read()
SRC_LAT = open(os.path.join(ROOT, "oracle", "lattice.py")).read()

D2 = dict(lat=L.D2Q9)

# (slip, expression, planted form, pin module, pin test, its arguments)
CASES = [
    ("gradient halved", "return gr / (2.0 * T)", "return gr / (4.0 * T)",
     "test_oracle_stencil", "test_linear_and_quadratic_exactness", D2),
    ("Laplacian factor 2 dropped", "return 2.0 * lap / T", "return lap / T",
     "test_oracle_stencil", "test_fourier_symbols", dict(lat=L.D2Q9, axis=0)),
    ("wall reads wrap around", "idx = np.clip(idx, 0, n - 1)", "idx = idx % n",
     "test_oracle_stencil", "test_wall_nodes_read_the_adjacent_fluid_value", dict(lat=L.D3Q19, axis=1)),
    ("mu bulk root moved", "phi * (phi - 1.0) * (phi - 0.5)", "phi * (phi - 1.0) * (phi - 0.4)",
     "test_oracle_moments", "test_chemical_potential_vanishes_on_flat_profile", {}),
    ("mu gradient term sign", "- 1.5 * p.sigma * p.W * lap", "+ 1.5 * p.sigma * p.W * lap",
     "test_oracle_moments", "test_chemical_potential_vanishes_on_flat_profile", {}),
    ("1/tau_mix phases swapped", "1.0 / p.tau_L + pc * (1.0 / p.tau_H - 1.0 / p.tau_L)",
     "1.0 / p.tau_H + pc * (1.0 / p.tau_L - 1.0 / p.tau_H)",
     "test_oracle_moments", "test_tau_mix_interpolation", {}),
    ("tau from nu times T", "return self.nu_L / T + 0.5", "return self.nu_L * T + 0.5",
     "test_oracle_moments", "test_tau_mix_interpolation", {}),
    ("theta over 2W", "(1.0 - 4.0 * (phi - 0.5) ** 2) / p.W", "(1.0 - 4.0 * (phi - 0.5) ** 2) / (2.0 * p.W)",
     "test_oracle_moments", "test_h_equilibrium_moments", D2),
    ("normal regulariser 1e-3", "grad / (mag + p.eps)", "grad / (mag + 1e-3)",
     "test_oracle_moments", "test_h_equilibrium_moments", D2),
    ("h^eq theta term sign", "phi * G[i] + th * lat.w[i] * cn", "phi * G[i] - th * lat.w[i] * cn",
     "test_oracle_moments", "test_h_equilibrium_moments", D2),
    ("Gamma linear term halved", "1.0 + cu / T + cu ** 2", "1.0 + cu / (2.0 * T) + cu ** 2",
     "test_oracle_moments", "test_gamma_moments", D2),
    ("Gamma quadratic term 1/(2T)", "cu ** 2 / (2.0 * T * T)", "cu ** 2 / (2.0 * T)",
     "test_oracle_moments", "test_gamma_moments", D2),
    ("Gamma u^2 term 1/(2T^2)", "- usq / (2.0 * T)", "- usq / (2.0 * T * T)",
     "test_oracle_moments", "test_gamma_moments", D2),
    ("K_i Gamma - w to Gamma", "(G[i] - lat.w[i]) * p.rho_dif", "G[i] * p.rho_dif",
     "test_oracle_moments", "test_forcing_moments", D2),
    ("K_i mu term weight", "G[i] * mu / T", "lat.w[i] * mu / T",
     "test_oracle_moments", "test_forcing_moments", D2),
    ("K_i force term weight", "+ G[i] * cmu_F / T", "+ lat.w[i] * cmu_F / T",
     "test_oracle_moments", "test_forcing_moments", D2),
    ("K_i c - u to c", "(lat.c[i][a] - u[a]) * grad[a]", "lat.c[i][a] * grad[a]",
     "test_oracle_moments", "test_forcing_moments", D2),
    ("g^eq K_i/2 sign", "lat.w[i] * (P / T - rho) - 0.5 * K[i]", "lat.w[i] * (P / T - rho) + 0.5 * K[i]",
     "test_oracle_moments", "test_g_equilibrium_moments", dict(lat=L.D2Q9, hocorr=True)),
    ("delta f^eq over 2T", "lat.w[i] * cu * lap_rho / (4.0 * T)", "lat.w[i] * cu * lap_rho / (2.0 * T)",
     "test_oracle_moments", "test_high_order_correction_moments", D2),
    ("velocity: force counted twice", "J += 0.5 * (mu[None] * grad + F)", "J += (mu[None] * grad + F)",
     "test_oracle_moments", "test_init_macro_roundtrip", dict(lat=L.D2Q9, force_mode=0)),
    ("velocity: lap rho / 2", "rho + 0.25 * p.rho_dif * lap", "rho + 0.5 * p.rho_dif * lap",
     "test_oracle_moments", "test_init_macro_roundtrip", dict(lat=L.D2Q9, force_mode=0)),
    ("pressure u . grad phi sign", "+ 0.5 * T * p.rho_dif", "- 0.5 * T * p.rho_dif",
     "test_oracle_moments", "test_init_macro_roundtrip", dict(lat=L.D2Q9, force_mode=0)),
    ("pressure from u = 0", "P = pressure(g, u, grad, p)", "P = pressure(g, 0 * u, grad, p)",
     "test_oracle_moments", "test_init_macro_roundtrip", dict(lat=L.D2Q9, force_mode=0)),
    ("Phi_i trace without T", "(ccPi - T * trace)", "(ccPi - trace)",
     "test_oracle_moments", "test_hermite_filter", D2),
    ("Phi_i over 2T", "lat.w[i] / (2.0 * T * T)", "lat.w[i] / (2.0 * T)",
     "test_oracle_moments", "test_hermite_filter", D2),
    ("Pi with c instead of c c", "Pi[a, b] += c[a] * c[b] * f[l]", "Pi[a, b] += c[a] * f[l]",
     "test_oracle_moments", "test_filtered_equals_bgk_on_hermite_nonequilibrium", D2),
    ("filter relaxes at omega/2", "(1.0 - omega)[None]", "(1.0 - 0.5 * omega)[None]",
     "test_oracle_moments", "test_filtered_equals_bgk_on_hermite_nonequilibrium", D2),
    ("BGK collision without K_i", "gstar = g - (g - geq) * omega[None] + K", "gstar = g - (g - geq) * omega[None]",
     "test_oracle_moments", "test_filtered_equals_bgk_on_hermite_nonequilibrium", D2),
    ("filtered collision without K_i", "gstar = geq + K + (1.0 - omega)", "gstar = geq + (1.0 - omega)",
     "test_oracle_moments", "test_collision_moments", D2),
    ("Chapman-Enskog without transpose", "(du + np.swapaxes(du, 0, 1))", "(2.0 * du)",
     "test_oracle_moments", "test_chapman_enskog_rebuild", {}),
    ("Chapman-Enskog with tau - 1/2", "coef = -tau * T * density(phi, p)",
     "coef = -(tau - 0.5) * T * density(phi, p)",
     "test_oracle_moments", "test_chapman_enskog_rebuild", {}),
    ("h relaxes with tau + 1/2", "h - (h - heq) / p.tau_phi", "h - (h - heq) / (p.tau_phi + 0.5)",
     "test_oracle_physics", "test_diffusion_rate_is_mobility", dict(lat=L.D2Q9, shape=(1, 1, 128))),
    ("tau_phi offset 0.6", "return self.M / T + 0.5", "return self.M / T + 0.6",
     "test_oracle_physics", "test_diffusion_rate_is_mobility", dict(lat=L.D2Q9, shape=(1, 1, 128))),
    ("bounce-back keeps direction", "back = fstar[lat.opp[i]] if", "back = fstar[i] if",
     "test_oracle_physics", "test_global_conservation", dict(lat=L.D2Q9, shape=(1, 13, 17), walls=True)),
    ("moving-wall term halved", "term[j] = 2.0 * lat.w[j] * s * cu / T", "term[j] = lat.w[j] * s * cu / T",
     "test_oracle_physics", "test_single_phase_couette_is_linear", {}),
    ("moving-wall g term with phi", "moving_wall_terms(lat, p, density(phi, p), shape)",
     "moving_wall_terms(lat, p, phi, shape)",
     "test_oracle_units", "test_density_scaling_symmetry", dict(name="D2Q9 sliding wall, delta theta")),
    ("buoyancy about rho_L", "g * (rho - p.rho_bar)[None]", "g * (rho - p.rho_L)[None]",
     "test_oracle_physics", "test_buoyancy_force_has_no_net_push", dict(lat=L.D2Q9, shape=(1, 20, 26))),
    ("rho_bar of 1 - phi", "return p.rho_L + p.rho_dif * float(phi.mean())",
     "return p.rho_H - p.rho_dif * float(phi.mean())",
     "test_oracle_physics", "test_buoyancy_force_has_no_net_push", dict(lat=L.D2Q9, shape=(1, 20, 26))),
    ("hydrostatic trapezoid half dropped", "- 0.5 * F - 0.5 * np.take(F, [0], axis=axis)",
     "- 0.5 * np.take(F, [0], axis=axis)",
     "test_oracle_physics", "test_hydrostatic_start_balances_the_body_force", {}),
    ("delta theta gate sign", "np.maximum(0.0, (2.0 * phi - 1.0) * lap)", "np.maximum(0.0, (1.0 - 2.0 * phi) * lap)",
     "test_oracle_dtheta", "test_vanishes_on_tanh_profile", dict(W=2.5, offset=0.0)),
]


def _planted(old, new, src=SRC, fname="pflbm.py"):
    assert src.count(old) == 1, f"the expression must occur once: {old!r}"
    name = "oracle._planted_" + fname[:-3]
    mod = types.ModuleType(name)
    mod.__package__ = "oracle"
    mod.__file__ = os.path.join(ROOT, "oracle", fname)
    sys.modules[name] = mod        # dataclasses resolve their module while the class is built
    try:
        exec(compile(src.replace(old, new), mod.__file__, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


@pytest.mark.parametrize("slip,old,new,pin_module,pin,kwargs", CASES, ids=[c[0] for c in CASES])
def test_pin_fails_on_planted_slip(monkeypatch, slip, old, new, pin_module, pin, kwargs):
    tm = importlib.import_module(pin_module)
    test = getattr(tm, pin)
    test(**kwargs)                                  # the pin holds on the oracle as it is
    monkeypatch.setattr(tm, "O", _planted(old, new))
    with pytest.raises(AssertionError):
        test(**kwargs)


# surrogate network oracle: (slip, expression, planted form, pin test of test_oracle_surrogate, arguments)
SG_CASES = [
    ("conv reads p - d", "xs = np.roll(x, shift=(1 - dy, 1 - dx), axis=(1, 2))\n            out +=",
     "xs = np.roll(x, shift=(dy - 1, dx - 1), axis=(1, 2))\n            out +=", "test_conv_matches_loop_definition", {}),
    ("conv taps transposed", 'out += np.einsum("nhwi,oi->nhwo", xs, W[:, :, dy, dx])',
     'out += np.einsum("nhwi,oi->nhwo", xs, W[:, :, dx, dy])', "test_conv_matches_loop_definition", {}),
    ("input gradient shifted the wrong way", "shift=(dy - 1, dx - 1), axis=(1, 2))",
     "shift=(1 - dy, 1 - dx), axis=(1, 2))", "test_conv_backward_finite_differences", {}),
    ("weight gradient taps transposed", 'gW[:, :, dy, dx] = np.einsum("nhwo,nhwi->oi", gout, xs)',
     'gW[:, :, dx, dy] = np.einsum("nhwo,nhwi->oi", gout, xs)', "test_conv_backward_finite_differences", {}),
    ("pooling gradient not divided by f^2", "return np.repeat(np.repeat(g, f, axis=1), f, axis=2) / (f * f)",
     "return np.repeat(np.repeat(g, f, axis=1), f, axis=2)", "test_pool_and_upsample_adjoints", dict(f=2)),
    ("upsampling gradient averaged", "return g.reshape(N, H // f, f, W // f, f, C).sum(axis=(2, 4))",
     "return g.reshape(N, H // f, f, W // f, f, C).mean(axis=(2, 4))", "test_pool_and_upsample_adjoints", dict(f=2)),
    ("skip-connection gradient dropped", 'gs3 = gs3 + pool_backward(layer_back("b", ghb))',
     'gs3 = pool_backward(layer_back("b", ghb))', "test_network_gradient_finite_differences", {}),
    ("ReLU gradient unmasked", "ga = gy * (cache[name] > 0)", "ga = gy", "test_network_gradient_finite_differences", {}),
    ("concatenation split swapped", "gs1, gt2 = gc1[..., :n1], upsample_backward(gc1[..., n1:])",
     "gs1, gt2 = gc1[..., n1:], upsample_backward(gc1[..., :n1])", "test_network_gradient_finite_differences", {}),
    ("loss gradient factor 2 dropped", "gout = 2.0 * (out - target) / out.size", "gout = (out - target) / out.size",
     "test_network_gradient_finite_differences", {}),
    ("residual branch dropped", "return x + delta, c", "return delta, c", "test_identity_when_last_layer_is_zero", {}),
]


@pytest.mark.parametrize("slip,old,new,pin,kwargs", SG_CASES, ids=[c[0] for c in SG_CASES])
def test_surrogate_pin_fails_on_planted_slip(monkeypatch, slip, old, new, pin, kwargs):
    tm = importlib.import_module("test_oracle_surrogate")
    test = getattr(tm, pin)
    test(**kwargs)
    monkeypatch.setattr(tm, "S", _planted(old, new, SRC_SG, "surrogate.py"))
    with pytest.raises(AssertionError):
        test(**kwargs)


# validation diagnostics: (slip, expression, planted form, pin test of test_oracle_diagnostics, arguments)
DG_CASES = [
    ("3-D radius with the 2-D formula", "return (3.0 * V / (4.0 * np.pi)) ** (1.0 / 3.0)",
     "return (V / np.pi) ** (1.0 / 3.0)", "test_effective_radius_of_a_tanh_sphere",
     dict(dim=3, R=9.6, drop=True)),
    ("bubble volume from phi", "V = float(phi.sum()) if drop else float((1.0 - phi).sum())",
     "V = float(phi.sum())", "test_effective_radius_of_a_tanh_sphere", dict(dim=2, R=11.7, drop=False)),
    ("jump outside minus inside", "return float(inside - outside)", "return float(outside - inside)",
     "test_laplace_jump_of_a_step_field", {}),
    ("distance without minimum image", "dd = (dd + n / 2.0) % n - n / 2.0", "dd = dd % n",
     "test_radial_distance_minimum_image", {}),
]


@pytest.mark.parametrize("slip,old,new,pin,kwargs", DG_CASES, ids=[c[0] for c in DG_CASES])
def test_diagnostics_pin_fails_on_planted_slip(monkeypatch, slip, old, new, pin, kwargs):
    tm = importlib.import_module("test_oracle_diagnostics")
    test = getattr(tm, pin)
    test(**kwargs)
    monkeypatch.setattr(tm, "D", _planted(old, new, SRC_DG, "diagnostics.py"))
    with pytest.raises(AssertionError):
        test(**kwargs)


# velocity sets: (slip, expression, planted form, lattice, pin test of test_oracle_lattice)
LAT_CASES = [
    ("D3Q19 edge pair made corners", "(1, 0, 1), (-1, 0, -1)", "(1, 1, 1), (-1, -1, -1)", "D3Q19",
     "test_velocity_set_matches_definition"),
    ("D3Q19 edge weight 1/18", "[1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12",
     "[1.0 / 3.0] + [1.0 / 18.0] * 7 + [1.0 / 36.0] * 11", "D3Q19", "test_isotropy"),
    ("D2Q9 rest weight 1/3", "[4.0 / 9.0] + [1.0 / 9.0] * 4", "[1.0 / 3.0] + [1.0 / 9.0] * 4", "D2Q9",
     "test_isotropy"),
    ("D2Q9 diagonal pair made long axis", "(1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)",
     "(2, 0, 0), (-1, 1, 0), (-2, 0, 0), (1, -1, 0)", "D2Q9", "test_velocity_set_matches_definition"),
]


@pytest.mark.parametrize("slip,old,new,name,pin", LAT_CASES, ids=[c[0] for c in LAT_CASES])
def test_lattice_pin_fails_on_planted_slip(slip, old, new, name, pin):
    tm = importlib.import_module("test_oracle_lattice")
    test = getattr(tm, pin)
    test(lat=getattr(L, name))
    planted = _planted(old, new, SRC_LAT, "lattice.py")
    with pytest.raises(AssertionError):
        test(lat=getattr(planted, name))
