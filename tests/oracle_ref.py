"""Oracle-side helpers for the parity tests (calls only oracle/ and workloads/)."""
import numpy as np

from oracle.assemble import Assembly, pml_sigma
from oracle.mesh import Mesh
from oracle.solver import Solver


def sigma_of(mesh, pml):
    if pml is None:
        return None
    return pml_sigma(mesh.centroids(), pml["lo"], pml["hi"], pml["thickness"],
                     pml["sigma_max"], pml.get("order", 2))


def build(xyz, tets, p, eps, mu, flux, pml=None, rows=None, S=1, sources=None, mesh=None):
    m = mesh or Mesh(xyz, tets)
    asm = Assembly(m, p, eps, mu, flux, sigma=sigma_of(m, pml), rows=rows)
    return Solver(asm, S=S, sources=sources)


def rhs(solver, u, aux=None, t=0.0):
    """Oracle du/dt for state u (K, S, 6, N) [+ aux] -> (du rows, daux rows or None)."""
    y = solver.rhs(solver.pack(u, aux), t)
    return solver.unpack(y)


def rel_err(got, ref):
    """max-norm error relative to the max-norm of the reference."""
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def rel_l2(got, ref):
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))
