"""Pin of the oracle's incident-field faces (Sec. V: the 3-D source is an
incident plane wave; Appendix A sets the boundary value of e to 2 E_inc + e).

A TEM pulse E = x g(t - z), H = y g(t - z) between two conducting plates (x = 0,
0.5: E normal to them) is injected through the face z = 0 of a slab that is
long in y, so the two side walls (which a plane wave does not satisfy) are
further from the compared region than the pulse has travelled.  Before the
pulse reaches the far wall, E and H in the middle of the slab must be the
analytic pulse: with the upwind flux the oracle is within 2 % at a 4^3 grid,
p = 2 (0.5 % at 6^3), and the injected amplitude within 0.2 %.  A missing
factor of 2, a wrong sign of the ghost state, or h+ = +h- (no boundary
condition at all: the run grows without bound) fail it.
"""
import math

import numpy as np

import workloads as W
from oracle.assemble import Assembly
from oracle.mesh import Mesh
from oracle.solver import Solver


def test_tem_pulse_enters_through_the_incident_face():
    n, p = 4, 2
    lo, hi = (0, -1, 0), (0.5, 1.5, 1)
    xyz, tets = W.kuhn_mesh(n, lo, hi)
    m = Mesh(xyz, tets)
    faces = [np.delete(m.tets[T], f) for T in range(m.K) for f in range(4)
             if m.nbr[T, f] < 0 and np.all(np.abs(xyz[np.delete(m.tets[T], f), 2]) < 1e-12)]
    assert len(faces) == 2 * n * n
    a = Assembly(m, p, 1.0, 1.0, "upwind", incident=faces)
    s = Solver(a)
    sig, t0, T = 0.15, 0.6, 1.0
    s.set_incident((1, 0, 0), (0, 0, 1), 1.0, 0.0, 1.0 / (2 * math.pi * sig), t0)
    dt = 0.3 * min((np.array(hi) - np.array(lo)) / n) / (p + 1) ** 2
    steps = int(round(T / dt))
    u = s.unpack(s.lsrk4(np.zeros((a.ndof, 1)), 0.0, T / steps, steps))[0][:, 0]
    g = lambda r: np.exp(-(T - t0 - r[:, 2]) ** 2 / (2 * sig * sig))
    ex = s.project(lambda r: np.stack([g(r), 0 * g(r), 0 * g(r)], axis=1), "E")
    hy = s.project(lambda r: np.stack([0 * g(r), g(r), 0 * g(r)], axis=1), "E")
    mid = (m.centroids()[:, 1] > 0.0) & (m.centroids()[:, 1] < 0.5)
    e_err = np.linalg.norm(u[mid, 0:3] - ex[mid]) / np.linalg.norm(ex[mid])
    h_err = np.linalg.norm(u[mid, 3:6] - hy[mid]) / np.linalg.norm(hy[mid])
    amp = np.linalg.norm(u[mid, 0:3]) / np.linalg.norm(ex[mid])
    assert e_err < 0.03 and h_err < 0.03, (e_err, h_err)
    assert abs(amp - 1.0) < 0.01, amp
