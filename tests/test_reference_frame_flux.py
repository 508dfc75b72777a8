"""The algebra behind the stage kernel's reference-frame flux (no GPU).

The pulled-back flux g = 2|F| A^-1 flux of the central/upwind flux (Eqs. (uwc),
(cwc); PEC ghost state of Sec. IV) is written in the kernel from the reference
jumps dx = Q x+ - alpha x- with Q = A^T A_n^-T, through the identity
(M a) x (M b) = det M M^-T (a x b) for M = A^-T.  These tests restate both forms
with numpy on random element maps (both orientations), every face, interior and
PEC faces, central and upwind coefficients, and check that they agree, that the
axis faces' short forms (cross products as permutations) agree too, and that
the component the kernel neither lifts nor traces is zero in the physical form."""
import numpy as np
import pytest

# reference face normals scaled by twice the face area: faces 0..3 of the unit tet
M_F = [np.array([1.0, 1.0, 1.0]), np.array([-1.0, 0.0, 0.0]),
       np.array([0.0, -1.0, 0.0]), np.array([0.0, 0.0, -1.0])]


def physical_form(A, An, f, xe, ye, xh, yh, ce, be, ch, bh, pec):
    """g_E, g_H from physical traces X = A^-T x on each side (PEC: e+ = -e-, h+ = h-)."""
    M, Mn = np.linalg.inv(A).T, np.linalg.inv(An).T
    v = M @ M_F[f]
    n = v / np.linalg.norm(v)
    two_f = abs(np.linalg.det(A)) * np.linalg.norm(v)
    em, hm = M @ xe, M @ xh
    ep, hp = (-em, hm) if pec else (Mn @ ye, Mn @ yh)
    de, dh = ep - em, hp - hm
    fe = ce * np.cross(n, dh) - be * np.cross(n, np.cross(n, de))
    fh = ch * np.cross(n, de) + bh * np.cross(n, np.cross(n, dh))
    return two_f * np.linalg.inv(A) @ fe, -two_f * np.linalg.inv(A) @ fh


def reference_form(A, An, f, xe, ye, xh, yh, ce, be, ch, bh, pec):
    """The same fluxes from reference-frame jumps only (no map of either trace)."""
    M = np.linalg.inv(A).T
    Q = np.eye(3) if pec else A.T @ np.linalg.inv(An).T
    ae, ah = (2.0, 0.0) if pec else (1.0, 1.0)
    yE = np.zeros(3) if pec else ye
    yH = np.zeros(3) if pec else yh
    de = Q @ yE - ae * xe
    dh = Q @ yH - ah * xh
    m = M_F[f]
    st = np.sign(np.linalg.det(A))
    k = 1.0 / (abs(np.linalg.det(A)) * np.linalg.norm(M @ m))
    G = A.T @ A
    ge = st * ce * np.cross(m, dh) - k * be * np.cross(m, G @ np.cross(m, de))
    gh = -st * ch * np.cross(m, de) - k * bh * np.cross(m, G @ np.cross(m, dh))
    return ge, gh, de, dh, st, k, G


def axis_short_form(f, de, dh, st, k, G, ce, be, ch, bh):
    """Face a + 1 (m = -e_a): (m x y)_a = 0, (m x y)_b = y_c, (m x y)_c = -y_b with
    (a, b, c) cyclic; only components b and c of the jumps enter."""
    a = f - 1
    b, c = (a + 1) % 3, (a + 2) % 3
    ge, gh = np.zeros(3), np.zeros(3)
    ge[b] = st * ce * dh[c] - k * be * (G[c, b] * de[c] - G[c, c] * de[b])
    ge[c] = -st * ce * dh[b] - k * be * (-G[b, b] * de[c] + G[b, c] * de[b])
    gh[b] = -st * ch * de[c] - k * bh * (G[c, b] * dh[c] - G[c, c] * dh[b])
    gh[c] = st * ch * de[b] - k * bh * (-G[b, b] * dh[c] + G[b, c] * dh[b])
    return ge, gh


def _cases():
    rng = np.random.default_rng(2002)
    for trial in range(40):
        A = rng.standard_normal((3, 3)) + 2 * np.eye(3)
        An = rng.standard_normal((3, 3)) + 2 * np.eye(3)
        if trial % 2:
            A[:, 0] *= -1.0          # the other orientation, s_T = -1
        for f in range(4):
            for pec in (False, True):
                for upwind in (False, True):
                    zm, zp = rng.uniform(0.5, 2.0, 2)
                    if upwind:
                        coef = (zp / (zm + zp), 1 / (zm + zp), zm / (zm + zp), zm * zp / (zm + zp))
                    else:
                        coef = (0.5, 0.0, 0.5, 0.0)
                    x = [rng.standard_normal(3) for _ in range(4)]
                    yield A, An, f, x, coef, pec


def test_reference_form_equals_physical_form():
    worst = 0.0
    for A, An, f, (xe, ye, xh, yh), coef, pec in _cases():
        ge0, gh0 = physical_form(A, An, f, xe, ye, xh, yh, *coef, pec)
        ge1, gh1, *_ = reference_form(A, An, f, xe, ye, xh, yh, *coef, pec)
        scale = max(np.abs(ge0).max(), np.abs(gh0).max())
        worst = max(worst, np.abs(ge1 - ge0).max() / scale, np.abs(gh1 - gh0).max() / scale)
    assert worst < 1e-11


def test_axis_faces_short_form_and_zero_component():
    for A, An, f, (xe, ye, xh, yh), coef, pec in _cases():
        if f == 0:
            continue
        ge0, gh0 = physical_form(A, An, f, xe, ye, xh, yh, *coef, pec)
        ge1, gh1, de, dh, st, k, G = reference_form(A, An, f, xe, ye, xh, yh, *coef, pec)
        scale = max(np.abs(ge0).max(), np.abs(gh0).max())
        # the pulled-back flux on face a + 1 has no component a ...
        a = f - 1
        assert abs(ge0[a]) < 1e-12 * scale and abs(gh0[a]) < 1e-12 * scale
        # ... and component a of the jumps (hence of the own trace) does not enter
        de_cut, dh_cut = de.copy(), dh.copy()
        de_cut[a] = dh_cut[a] = np.nan
        ge2, gh2 = axis_short_form(f, de_cut, dh_cut, st, k, G, *coef)
        assert np.all(np.isfinite(ge2)) and np.all(np.isfinite(gh2))
        assert np.abs(ge2 - ge0).max() < 1e-11 * scale
        assert np.abs(gh2 - gh0).max() < 1e-11 * scale


@pytest.mark.parametrize("f", [0, 1, 2, 3])
def test_physical_jump_from_reference_jump(f):
    """The adjoint's forward quantities are physical jumps; the kernel forms them
    as A^-T dx from the reference jumps it already has."""
    for A, An, ff, (xe, ye, xh, yh), coef, pec in _cases():
        if ff != f:
            continue
        M, Mn = np.linalg.inv(A).T, np.linalg.inv(An).T
        _, _, de, dh, *_ = reference_form(A, An, f, xe, ye, xh, yh, *coef, pec)
        de_phys = -2 * M @ xe if pec else Mn @ ye - M @ xe
        dh_phys = np.zeros(3) if pec else Mn @ yh - M @ xh
        assert np.allclose(M @ de, de_phys, rtol=1e-12, atol=1e-12)
        assert np.allclose(M @ dh, dh_phys, rtol=1e-12, atol=1e-12)
