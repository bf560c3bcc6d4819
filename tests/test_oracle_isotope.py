"""Pins of the isotope-scattering oracle (Eq. (isotope)): the completeness sum rule with a
flat delta (closed form), invariance under a rotation of the Cartesian frame (which fixes
where the Cartesian sum sits), linearity in g, and the mass-variance parameter."""
import math

import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _two_atom(rot=None):
    c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
    lat, pos = c.lattice, c.positions
    if rot is not None:
        lat, pos = lat @ rot.T, pos @ rot.T
    return P.Crystal(lat, pos, np.array([39.95, 83.8]), "fcc2")


def _phonons(c, mesh):
    f2 = P.ifc2_lj(c, P.LennardJones())
    q = O.grid.mesh_qred(mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    return freq, evec


def test_flat_delta_sum_rule_closed_form():
    """With delta -> constant c, completeness over (q', s') gives
    gamma_s = (pi/2) w_s^2 c sum_i g_i |e_i(s)|^2 (normalisation, w^2, per-atom weights)."""
    mesh = (3, 2, 2)
    freq, evec = _phonons(_two_atom(), mesh)
    g = np.array([0.1, 0.3])
    sig = 1e4
    irr = [1, 5]
    got = O.isotope.gamma_iso(freq, evec, irr, g, "gauss", sig, f_min=-1e9, window=1e9)
    c = 1.0 / (math.sqrt(math.pi) * sig) / (2 * math.pi)
    for k, iq in enumerate(irr):
        e = evec[iq].reshape(2, 3, -1)
        w = 2 * math.pi * freq[iq]
        ref = 0.5 * math.pi * w * w * c * np.einsum("i,ias->s", g, np.abs(e) ** 2)
        assert np.allclose(got[k], ref, rtol=1e-7, atol=0)


def test_rotation_of_the_frame_leaves_the_rate_unchanged():
    """A rotated crystal has rotated displacement patterns; the rate (degenerate-averaged)
    must not change (it would with the Cartesian sum outside the modulus)."""
    mesh = (3, 3, 2)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    g = np.array([0.2, 0.05])
    f0, e0 = _phonons(_two_atom(), mesh)
    f1, e1 = _phonons(_two_atom(Q), mesh)
    irr = list(range(0, 18, 3))
    g0 = O.isotope.gamma_iso(f0, e0, irr, g, "gauss", 0.3)
    g1 = O.isotope.gamma_iso(f1, e1, irr, g, "gauss", 0.3)
    assert g0.max() > 0
    for k, iq in enumerate(irr):
        a = O.anharmonic.degenerate_average(f0[iq], g0[k])
        b = O.anharmonic.degenerate_average(f1[iq], g1[k])
        assert np.abs(a - b).max() <= 1e-9 * g0.max()


def test_linear_in_g_and_mass_variance_parameter():
    mesh = (2, 2, 2)
    freq, evec = _phonons(_two_atom(), mesh)
    a = O.isotope.gamma_iso(freq, evec, [1], [0.1, 0.0])
    b = O.isotope.gamma_iso(freq, evec, [1], [0.0, 0.2])
    c = O.isotope.gamma_iso(freq, evec, [1], [0.3, 0.6])
    assert np.allclose(c, 3 * a + 3 * b, rtol=1e-12, atol=1e-300)
    # 50/50 Ar/Kr virtual crystal: mbar = 61.875, g = 0.5 (21.925/61.875)^2 * 2
    assert abs(O.isotope.g_factor([0.5, 0.5], [39.95, 83.8]) - (21.925 / 61.875) ** 2) < 1e-15
