"""QHGK conductivity of a Gamma-only cell on the GPU (phx_kappa_qhgk) against the oracle of
Eq. (qhgk) with shared eigenvectors: an ideal 3x3x3 supercell (exact degeneracies) and a
disordered 80-atom cell with GPU linewidths."""
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


def _gamma_point(ctx, c, f2):
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), np.zeros((1, 3)),
                                    want_vel=False, want_vv=False)
    return freq[0], evec[0]


def test_ideal_supercell_matches_oracle(ctx):
    sc = P.supercell(P.fcc_primitive(), (3, 3, 3))
    pot = P.LennardJones()
    s2 = P.ifc2_lj(sc, pot)
    D = O.gammapoint.dynmat(s2.idx, s2.val.reshape(-1, 9), sc.masses)
    lam, E = np.linalg.eigh(D)
    f = O.harmonic.frequencies_from_eigenvalues(lam)
    g = 0.08 + 0.25 * f ** 2
    k = ctx.kappa_qhgk(sc.lattice, sc.masses, sc.positions, s2.idx, s2.val.reshape(-1, 9), f,
                       E.astype(np.complex128), g, 60.0)
    ref = O.qhgk.kappa_gamma_cell(s2.idx, s2.val, sc.masses, sc.positions, sc.lattice, f, E, g, 60.0)
    assert np.abs(ref).max() > 0
    assert np.abs(k - ref).max() <= 1e-10 * np.abs(ref).max()


def test_disordered_cell_with_gpu_linewidths(ctx):
    c = P.random_masses(P.fcc_primitive_multiple(5.26, (5, 4, 4)), 39.95, 83.8, seed=11)
    rng = np.random.default_rng(11)
    c.positions = c.positions + rng.normal(scale=0.05, size=c.positions.shape)
    s2, s3 = P.ifc_lj_vectorised(c, P.LennardJones())
    f, E = _gamma_point(ctx, c, s2)
    h = ctx.fc3(c.lattice, c.masses, s3.idx, s3.val, (1, 1, 1))
    g = ctx.gamma_cell(h, f, E, 300.0, shape="lorentz", sigma=0.1, precision="fp64")
    k = ctx.kappa_qhgk(c.lattice, c.masses, c.positions, s2.idx, s2.val.reshape(-1, 9), f, E, g, 300.0)
    ref = O.qhgk.kappa_gamma_cell(s2.idx, s2.val, c.masses, c.positions, c.lattice, f, E.real, g, 300.0)
    assert np.trace(ref) > 0
    assert np.abs(k - ref).max() <= 1e-10 * np.abs(ref).max()
