"""Large-cell Gamma-point eigensolver (Householder + bisection + inverse iteration) against
the oracle's dynamical matrix solved by a library eigensolver, and against the primitive-cell
dispersion for an ideal supercell (exact degeneracies)."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_23728_gb300 as m
    c = m.Context(0)
    yield c
    c.close()


def _check(ctx, crystal, f2, ref_freq=None, orth_tol=1e-9):
    freq, evec, _, _ = ctx.harmonic(crystal.lattice, crystal.masses, f2.idx, f2.val.reshape(-1, 9),
                                    np.zeros((1, 3)), want_vel=False, want_vv=False)
    f = freq[0]
    E = evec[0]
    assert np.abs(E.imag).max() == 0.0
    Z = E.real
    D = O.gammapoint.dynmat(f2.idx, f2.val.reshape(-1, 9), crystal.masses)
    lam = np.linalg.eigvalsh(D)
    fo = np.sign(lam) * np.sqrt(np.abs(lam) * O.constants.EV_A2_AMU_TO_PS2) / O.constants.TWO_PI
    if ref_freq is not None:
        assert np.allclose(np.sort(ref_freq), fo, atol=1e-7)
    assert np.all(np.diff(f) >= 0)
    assert np.abs(f - fo).max() < 1e-6            # acoustic zeros are sqrt of rounding noise
    hi = fo > 0.05
    assert np.abs(f[hi] - fo[hi]).max() <= 1e-10 * fo.max()
    w2 = np.sign(f) * (f * O.constants.TWO_PI) ** 2 / O.constants.EV_A2_AMU_TO_PS2
    resid = np.abs(D @ Z - Z * w2).max() / np.abs(D).max()
    assert resid < 1e-11
    assert np.abs(Z.T @ Z - np.eye(Z.shape[0])).max() < orth_tol
    big = np.argmax(np.abs(Z), axis=0)
    assert np.all(Z[big, np.arange(Z.shape[1])] > 0)
    return f, Z


def test_ideal_supercell_exact_degeneracies(ctx):
    pot = P.LennardJones()
    sc = P.fcc_primitive_multiple(5.26, (6, 6, 6))
    s2, _ = P.ifc_lj_vectorised(sc, pot)
    prim = P.fcc_primitive()
    p2 = P.ifc2_lj(prim, pot)
    fm, _, _ = O.harmonic.solve(p2.idx, p2.val, prim.masses, prim.lattice, O.grid.mesh_qred((6, 6, 6)))
    _check(ctx, sc, s2, ref_freq=fm.ravel())


def test_disordered_ragged_cell(ctx):
    c = P.random_masses(P.fcc_primitive_multiple(5.26, (5, 4, 4)), 39.95, 83.8, seed=7)
    rng = np.random.default_rng(7)
    c.positions = c.positions + rng.normal(scale=0.05, size=c.positions.shape)
    s2, _ = P.ifc_lj_vectorised(c, P.LennardJones())
    _check(ctx, c, s2)


@pytest.mark.slow
def test_thousand_atom_cell(ctx):
    w = P.gamma_disordered_1000()
    s2, _ = P.ifc_lj_vectorised(w.crystal, w.pot)
    _check(ctx, w.crystal, s2)


def test_large_cell_rejects_non_gamma_and_velocities(ctx):
    import paper_2602_23728_gb300 as m
    c = P.fcc_primitive_multiple(5.26, (5, 4, 4))
    s2, _ = P.ifc_lj_vectorised(c, P.LennardJones())
    with pytest.raises(m.PhxError):
        ctx.harmonic(c.lattice, c.masses, s2.idx, s2.val.reshape(-1, 9), np.array([[0.5, 0.0, 0.0]]),
                     want_vel=False, want_vv=False)
    with pytest.raises(m.PhxError):
        ctx.harmonic(c.lattice, c.masses, s2.idx, s2.val.reshape(-1, 9), np.zeros((1, 3)))
