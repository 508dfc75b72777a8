"""Pins of the oracle against facts fixed by the paper and by mathematics.

P1  orthonormality of the reference basis, Eq. (ortho_cond); Jacobi
    polynomials against scipy's implementation.
P3  the at-most 3x3 block-diagonal mass matrix (abstract; Sec. II) and its
    closed-form inverse.
P4  geometry-free reference curl, Eq. (matrix_free_curl), and own-face
    terms, up to the orientation sign of the element map.
P5  central flux + PEC walls: skew-symmetric operator (energy conservation,
    Sec. III) and exact conservation of the staggered leapfrog energy.
P6  upwind flux: negative semidefinite symmetric part.
P8  PML tensors against the tables printed in Appendix A and against the
    complex stretching of Eq. (cartesian_stretching).
P9  the PML path with sigma = 0 reduces to the plain path.
P10 LSRK4 coefficients: fourth-order stability polynomial and order 4 on a
    non-autonomous problem.
P12 point source functional reproduces point evaluation of polynomial fields.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import eval_jacobi

import workloads as W
from oracle.assemble import Assembly, pml_eta_xi, pml_sigma
from oracle.basis import RefBasis, jacobi, tet_quadrature
from oracle.mesh import Mesh
from oracle.solver import LSRK4_A, LSRK4_B, LSRK4_C, Solver

HERE = os.path.dirname(__file__)


def _random_tets(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        V = rng.uniform(-1, 1, size=(4, 3))
        if abs(np.linalg.det(V[1:] - V[0])) > 0.05:
            out.append(V)
    return out


def test_p1_jacobi_matches_scipy():
    w = np.linspace(-1, 1, 11)
    for n in range(7):
        for a in (0.0, 1.0, 3.0, 7.0, 10.0):
            assert np.allclose(jacobi(n, a, 0.0, w), eval_jacobi(n, a, 0.0, w),
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_p1_gram_is_identity(p):
    b = RefBasis(p)
    pts, wq = tet_quadrature(p + 4)
    V = b.values(pts)
    G = (V * wq[:, None]).T @ V
    assert np.abs(G - np.eye(b.N)).max() < 1e-13
    assert b.N == W.n_modes(p)


def test_p1_gradients_against_finite_differences():
    b = RefBasis(3)
    pts = np.array([[0.1, 0.2, 0.3], [0.25, 0.05, 0.6], [0.4, 0.4, 0.1]])
    g = b.gradients(pts)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (b.values(pts + e) - b.values(pts - e)) / (2 * h)
        assert np.abs(fd - g[:, :, a]).max() < 1e-7


def _one_tet_mesh(V):
    return Mesh(V, np.array([[0, 1, 2, 3]]))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_p3_mass_is_3x3_block_diagonal(p):
    for V in _random_tets(5, 10 + p):
        m = _one_tet_mesh(V)
        a = Assembly(m, p, 2.5, 1.0)
        N = a.N
        M = 2.5 * a.M1[0]
        big = np.abs(M) > 1e-13 * np.abs(M).max()
        assert big.sum() <= 9 * N
        mask = np.kron(np.ones((3, 3)), np.eye(N)).astype(bool)
        assert not np.any(big & ~mask)
        A = m.A[0]
        Minv_closed = np.kron(A.T @ A / (2.5 * abs(m.det[0])), np.eye(N))
        assert np.allclose(np.linalg.inv(M), Minv_closed, rtol=1e-11,
                           atol=1e-11 * np.abs(Minv_closed).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_p4_curl_and_own_face_terms_are_geometry_free(p):
    ref = Assembly(_one_tet_mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])),
                   p, 1.0, 1.0)
    ref_faces = {e["f"]: e["x_own"] for e in ref.face}
    for V in _random_tets(6, 20 + p):
        m = _one_tet_mesh(V)
        a = Assembly(m, p, 1.0, 1.0)
        s = np.sign(m.det[0])
        scale = np.abs(ref.C_eh[0]).max()
        assert np.abs(a.C_eh[0] - s * ref.C_eh[0]).max() < 1e-12 * scale
        for e in a.face:
            assert np.abs(e["x_own"] - s * ref_faces[e["f"]]).max() < 1e-12 * scale


@pytest.mark.parametrize("n,p,jit", [(2, 2, 0.0), (2, 1, 0.15)])
def test_p5_central_pec_is_skew(n, p, jit):
    xyz, tets = W.kuhn_mesh(n, jitter=jit, seed=5)
    m = Mesh(xyz, tets)
    eps = W.lognormal_material(m.K, 2.0, 0.3, 1)
    a = Assembly(m, p, eps, 1.0, "central")
    K = a.Kmat.toarray()
    assert np.abs(K + K.T).max() <= 1e-13 * np.abs(K).max()


def test_p5_leapfrog_staggered_energy_is_conserved():
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=3)
    m = Mesh(xyz, tets)
    a = Assembly(m, 2, 1.0, 1.0, "central")
    s = Solver(a)
    u = W.random_state(a.K, 1, 2, seed=4)
    x = s.pack(u)
    nE = a.K * a.n3
    Me = a.M1
    hist = []

    def e_form(x1, x2, blk):
        v1 = x1[blk * nE:(blk + 1) * nE, 0].reshape(a.K, a.n3)
        v2 = x2[blk * nE:(blk + 1) * nE, 0].reshape(a.K, a.n3)
        return float(np.einsum("ki,kij,kj->", v1, Me, v2))

    prev = [x.copy()]

    def cb(n, t, xn):
        # W^n = E^n M E^n + H^{n-1/2} M H^{n+1/2}
        if len(prev) >= 1 and n >= 2:
            hist.append(e_form(xn, xn, 0) + e_form(prev[-1], xn, 1))
        prev.append(xn.copy())

    s.leapfrog(x, 0.0, 0.02, 60, callback=cb)
    hist = np.array(hist)
    assert np.abs(hist - hist[0]).max() < 1e-12 * abs(hist[0])


def test_p6_upwind_is_dissipative():
    xyz, tets = W.kuhn_mesh(2, jitter=0.15, seed=9)
    m = Mesh(xyz, tets)
    eps = W.sphere_material(xyz, tets, (0.5, 0.5, 0.5), 0.3, 4.0, 1.0)
    a = Assembly(m, 2, eps, 1.5, "upwind")
    K = a.Kmat.toarray()
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert ev.max() <= 1e-12 * np.abs(K).max()
    assert ev.min() < -1e-3     # genuinely dissipative


def test_p8_pml_tables_match_listing():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "pml_listing_tables.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        vals = np.array([float(v) for v in r[1:]])
        eta, xi = pml_eta_xi(vals[:3])
        assert np.array_equal(eta, vals[3:6]), r[0]
        assert np.array_equal(xi, vals[6:9]), r[0]


def test_p8_partial_fractions_match_complex_stretching():
    rng = np.random.default_rng(0)
    for _ in range(50):
        sig = rng.uniform(0, 10, 3) * (rng.uniform(size=3) < 0.7)
        omega = rng.uniform(0.1, 20)
        J = np.diag(1.0 + 1j * sig / omega)          # Jacobian of the stretching map
        Ji = np.linalg.inv(J)
        eps_t = np.linalg.det(J) * Ji @ Ji.T          # |A~| A~^-1 eps A~^-T, eps = 1
        lam = -1j * omega
        eta, xi = pml_eta_xi(sig)
        model = lam + eta + xi / (lam + sig)
        assert np.allclose(lam * np.diag(eps_t), model, rtol=1e-13, atol=1e-12)
        assert np.allclose(eps_t - np.diag(np.diag(eps_t)), 0)


def test_p8_pml_profile():
    c = np.array([[0.0, 0.0, 0.0], [0.875, 0.0, 0.0], [0.9, -0.95, 0.8]])
    s = pml_sigma(c, (-0.75,) * 3, (0.75,) * 3, 0.25, 40.0, 2)
    assert np.allclose(s[0], 0)
    assert np.allclose(s[1], [40 * 0.25, 0, 0])
    assert np.allclose(s[2], [40 * 0.36, 40 * 0.64, 40 * 0.04])


def test_p9_zero_sigma_reduces_to_plain_path():
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=1)
    m = Mesh(xyz, tets)
    plain = Assembly(m, 1, 1.0, 1.0, "upwind")
    withp = Assembly(m, 1, 1.0, 1.0, "upwind", sigma=np.zeros((m.K, 3)))
    u = W.random_state(m.K, 2, 1, seed=2)
    s0, s1 = Solver(plain, S=2), Solver(withp, S=2)
    r0 = s0.unpack(s0.rhs(s0.pack(u)))[0]
    r1, aux = s1.unpack(s1.rhs(s1.pack(u, np.zeros_like(u))))
    assert np.array_equal(r0, r1)
    assert np.all(aux == 0)


def _lsrk_step(f, y, t, dt):
    res = 0.0 * y
    for k in range(5):
        res = LSRK4_A[k] * res + dt * f(t + LSRK4_C[k] * dt, y)
        y = y + LSRK4_B[k] * res
    return y


def test_p10_lsrk4_stability_polynomial():
    zs = np.array([0.3, -0.7, 0.5j, -0.2 + 0.4j, 1.1, -1.3j])
    R = np.array([_lsrk_step(lambda t, y: z * y, 1.0 + 0j, 0.0, 1.0) for z in zs])
    V = np.vander(zs, 6, increasing=True)
    coef = np.linalg.solve(V, R)
    assert np.allclose(coef[:5], [1, 1, 0.5, 1 / 6, 1 / 24], atol=1e-12)
    assert abs(coef[5]) > 1e-4          # a genuine fifth-degree stage polynomial


def test_p10_lsrk4_order_four_non_autonomous():
    f = lambda t, y: np.cos(3 * t) * y + t ** 2
    from scipy.integrate import solve_ivp
    ref = solve_ivp(f, (0, 1), [1.0], rtol=1e-13, atol=1e-14).y[0, -1]
    errs = []
    for n in (20, 40, 80):
        y, t = np.array([1.0]), 0.0
        for _ in range(n):
            y = _lsrk_step(f, y, t, 1.0 / n)
            t += 1.0 / n
        errs.append(abs(y[0] - ref))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8)


def test_p12_point_source_reproduces_polynomial_point_values():
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=7)
    m = Mesh(xyz, tets)
    a = Assembly(m, 2, 1.0, 1.0)
    pos = np.array([0.37, 0.61, 0.29])
    d = np.array([0.2, -0.5, 1.0])
    s = Solver(a, S=1, sources=[dict(pos=pos, dir=d, f0=1.0, bw=1.0, t0=0.0)])
    _, T, w, _ = s.src[0]
    v = lambda r: np.stack([r[:, 0] * r[:, 1], 1 - r[:, 2] ** 2, r[:, 0] + 2 * r[:, 2]], axis=1)
    coef = s.project(v, "E")
    got = float(w @ coef[T].reshape(-1))
    assert abs(got - float(d @ v(pos[None, :])[0])) < 1e-12
