"""Element maps and face matching of the oracle (test infrastructure only).

Element map, Eq. (mapping_template): r = A_T r_hat + b_T with the columns of
A_T the edges v1-v0, v2-v0, v3-v0.  Convention shared with the CUDA path (a
convention, not code): the local vertex order of each tetrahedron is its
global vertex ids in ascending order, so that modal coefficients of both
implementations refer to the same mapped basis.

Neighbours are found *geometrically*: two faces match when their three
vertex coordinates coincide (rounded to 1e-12).  Outward normals come from
the face's cross product, oriented away from the opposite vertex.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, xyz, tets):
        xyz = np.asarray(xyz, dtype=np.float64)
        tets = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
        self.xyz = xyz
        self.tets = tets
        self.K = tets.shape[0]
        V = xyz[tets]                       # [K, 4, 3]
        self.verts = V
        self.b = V[:, 0, :].copy()
        self.A = np.stack([V[:, 1] - V[:, 0], V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]], axis=2)
        self.det = np.linalg.det(self.A)
        if np.any(np.abs(self.det) < 1e-300):
            raise ValueError("degenerate element")
        self.Ainv = np.linalg.inv(self.A)
        self._match_faces()

    def to_ref(self, T, r):
        """Physical points r [n, 3] of element T -> reference coordinates."""
        return (r - self.b[T][None, :]) @ self.Ainv[T].T

    def face_vertices(self, T, f):
        """Physical vertices of the face of T opposite local vertex f, and that vertex."""
        idx = [v for v in range(4) if v != f]
        return self.verts[T, idx, :], self.verts[T, f, :]

    def _match_faces(self):
        # key of a face: its three vertex coordinates, rounded, in lexicographic order
        F = np.stack([self.verts[:, [v for v in range(4) if v != f], :] for f in range(4)],
                     axis=1)                               # [K, 4, 3 verts, 3 coords]
        F = np.round(F, 12).reshape(-1, 3, 3)
        order = np.lexsort((F[:, :, 2], F[:, :, 1], F[:, :, 0]), axis=-1)
        F = np.take_along_axis(F, order[:, :, None], axis=1).reshape(-1, 9)
        _, inv, counts = np.unique(F, axis=0, return_inverse=True, return_counts=True)
        if np.any(counts > 2):
            raise ValueError("non-manifold face")
        self.nbr = -np.ones((self.K, 4), dtype=np.int64)
        srt = np.argsort(inv, kind="stable")
        inv_s = inv[srt]
        same = np.nonzero(inv_s[1:] == inv_s[:-1])[0]
        a, b = srt[same], srt[same + 1]
        self.nbr.reshape(-1)[a] = b // 4
        self.nbr.reshape(-1)[b] = a // 4

    def face_frame(self, T, f):
        """(P [3,3] face vertices, outward unit normal n, area)."""
        P, opp = self.face_vertices(T, f)
        c = np.cross(P[1] - P[0], P[2] - P[0])
        area = 0.5 * np.linalg.norm(c)
        n = c / np.linalg.norm(c)
        if np.dot(n, P[0] - opp) < 0:
            n = -n
        return P, n, area

    def locate(self, r, tol=1e-12):
        """Lowest-index element containing point r (barycentric >= -tol)."""
        for T in range(self.K):
            rh = self.to_ref(T, r[None, :])[0]
            lam = np.array([1.0 - rh.sum(), rh[0], rh[1], rh[2]])
            if np.all(lam >= -tol):
                return T
        raise ValueError("point outside mesh")

    def centroids(self):
        return self.verts.mean(axis=1)
