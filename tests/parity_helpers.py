"""Shared helpers of the GPU parity tests: run the same seeded case through
the CUDA library (C-ABI via the ctypes binding) and through the oracle,
and map between the two velocity orders by velocity vector."""
import numpy as np

from oracle import lattice as OL
from oracle import pflbm as O


def oracle_lattice(lat_id):
    return OL.D2Q9 if lat_id == 0 else OL.D3Q19


def oracle_params(prm, bc_user, lat_id):
    """Oracle Params equal to an lbm_params struct; bc_user per user axis."""
    names = {0: "periodic", 1: "wall"}
    bc = [names[b] for b in bc_user] + ["periodic"] * (3 - len(bc_user))
    if lat_id == 0:
        bc = [bc[0], bc[1], "periodic"]
    return O.Params(M=prm.M, W=prm.W, sigma=prm.sigma, rho_L=prm.rho_L, rho_H=prm.rho_H,
                    nu_L=prm.nu_L, nu_H=prm.nu_H, g=(prm.g[0], prm.g[1], prm.g[2] if lat_id == 1 else 0.0),
                    force_mode=prm.force_mode, eps=prm.eps, hocorr=bool(prm.hocorr),
                    modified_velocity=bool(prm.hocorr), bc=tuple(bc), C_dtheta=prm.C_dtheta)


def order_map(lat_id):
    """perm[k] = oracle index of the library's k-th velocity."""
    from paper_1812_00118_gb300 import lbm
    c, _ = lbm.lattice_info(lat_id)
    olat = oracle_lattice(lat_id)
    idx = {tuple(int(a) for a in v): i for i, v in enumerate(olat.c)}
    return np.array([idx[tuple(v)] for v in c.tolist()])


def lib_to_oracle_pops(flat, lat_id, shape):
    """Library populations (Q*N, library order) -> oracle (Q, nz, ny, nx)."""
    perm = order_map(lat_id)
    Q = len(perm)
    a = flat.reshape(Q, *shape)
    out = np.empty_like(a)
    out[perm] = a
    return out


def oracle_to_lib_pops(pops, lat_id):
    perm = order_map(lat_id)
    return np.ascontiguousarray(pops[perm]).reshape(-1)


def user_velocity(u3, lat_id):
    """Oracle velocity (3, nz, ny, nx) -> library layout (dim*N,)."""
    dim = 2 if lat_id == 0 else 3
    return np.ascontiguousarray(u3[:dim]).reshape(-1)


def oracle_macro_flat(h, g, lat, p, lat_id):
    m = O.macroscopic(h, g, lat, p)
    dim = 2 if lat_id == 0 else 3
    rho_u = (m["rho"][None] * m["u"])[:dim].reshape(-1)
    return m["phi"].reshape(-1), m["P"].reshape(-1), rho_u


def normwise(a, b):
    """max |a - b| / max |b| (reading: normwise error, u can be near zero)."""
    d = float(np.abs(np.asarray(a) - np.asarray(b)).max())
    s = float(np.abs(np.asarray(b)).max())
    return d / s if s > 0 else d
