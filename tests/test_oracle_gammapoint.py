"""Pins of the Gamma-only large-cell oracle (oracle.gammapoint) against the dense literal
evaluation of Eq. (phi3_proj), against the q-mesh linewidths through supercell folding, and of
its dynamical matrix against the primitive-cell dispersion; plus a check of the permutation
counting that a Gamma-only kernel may use (every unordered triple evaluated once)."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _disordered(mult=(3, 2, 2), seed=4, noise=0.05):
    c = P.random_masses(P.fcc_primitive_multiple(5.26, mult), 39.95, 83.8, seed=seed)
    rng = np.random.default_rng(seed)
    c.positions = c.positions + rng.normal(scale=noise, size=c.positions.shape)
    pot = P.LennardJones()
    return c, P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)


def _solve(c, f2):
    D = O.gammapoint.dynmat(f2.idx, f2.val.reshape(-1, 9), c.masses)
    lam, E = np.linalg.eigh(D)
    f = np.sign(lam) * np.sqrt(np.abs(lam) * O.constants.EV_A2_AMU_TO_PS2) / O.constants.TWO_PI
    return f, E


@pytest.mark.parametrize("shape", ["lorentz", "gauss"])
def test_gamma_modes_equals_dense_literal(shape):
    """Sparse per-mode evaluation == dense einsum of Eq. (phi3_proj) over the full tensor
    (catches a wrong contraction index, a missing mass factor or image sum)."""
    c, f2, f3 = _disordered()
    D1 = O.gammapoint.dynmat(f2.idx, f2.val.reshape(-1, 9), c.masses)
    D2 = O.supercell.gamma_point_dynmat(f2.idx, f2.val, c.masses)
    assert np.abs(D1 - D2).max() <= 1e-13 * np.abs(D2).max()
    T, sig = 40.0, 0.3
    fs, gs = O.supercell.gamma_only(f2.idx, f2.val, f3.idx, f3.val, c.masses, T, shape, sig)
    f, E = _solve(c, f2)
    assert np.allclose(f, fs, atol=1e-6)          # acoustic zeros are ~1e-8 noise
    g = O.gammapoint.gamma_modes(f3.idx, f3.val, c.masses, f, E, range(f.shape[0]), T, shape, sig)
    assert gs.max() > 0
    assert np.abs(g - gs).max() <= 1e-11 * gs.max()


def test_gamma_modes_folds_to_mesh_lorentz():
    """Lorentzian form of the folding pin: mesh linewidths of the 1-atom cell on a 3x2x2 mesh
    (degenerate-averaged) equal the per-mode Gamma-only linewidths of the 3x2x2 supercell."""
    pot = P.LennardJones()
    c = P.fcc_primitive()
    mesh = (3, 2, 2)
    T, sig = 60.0, 0.3
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    q = O.grid.mesh_qred(mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    g = O.anharmonic.gamma(fc3, mesh, freq, evec, np.arange(q.shape[0]), T, "lorentz", sig)
    sc = P.supercell(c, mesh)
    s2, s3 = P.ifc2_lj(sc, pot), P.ifc3_lj(sc, pot)
    fs, E = _solve(sc, s2)
    gs = O.gammapoint.gamma_modes(s3.idx, s3.val, sc.masses, fs, E, range(fs.shape[0]), T, "lorentz", sig)
    fm, gm = freq.ravel(), g.ravel()
    tol = 1e-5 * np.abs(fs).max()
    used = 0
    for f in np.unique(np.round(fs, 6)):
        if f < 0.01:
            continue
        mm, ms = np.abs(fm - f) < tol, np.abs(fs - f) < tol
        assert mm.sum() == ms.sum()
        assert abs(gm[mm].mean() - gs[ms].mean()) <= 1e-10 * gs.max()
        used += 1
    assert used > 3 and gs.max() > 0


def test_large_cell_dynmat_folds_primitive_dispersion():
    """Gamma frequencies of an ideal 6x6x6 supercell (648 modes) = the primitive cell's
    frequencies on the 6x6x6 mesh (catches a wrong block placement or mass factor)."""
    pot = P.LennardJones()
    prim = P.fcc_primitive()
    sc = P.fcc_primitive_multiple(5.26, (6, 6, 6))
    s2, _ = P.ifc_lj_vectorised(sc, pot)
    fs, E = _solve(sc, s2)
    p2 = P.ifc2_lj(prim, pot)
    q = O.grid.mesh_qred((6, 6, 6))
    fm, _, _ = O.harmonic.solve(p2.idx, p2.val, prim.masses, prim.lattice, q)
    assert np.allclose(np.sort(fm.ravel()), fs, atol=1e-7)
    assert np.abs(E.T @ E - np.eye(E.shape[0])).max() < 1e-12


def test_vectorised_ifcs_equal_reference_builder():
    """The vectorised large-cell IFC builder gives the same entries as the reference builder."""
    c, f2, f3 = _disordered((2, 2, 1), seed=1)
    b2, b3 = P.ifc_lj_vectorised(c, P.LennardJones())
    o = np.lexsort(f3.idx.T[::-1])
    p = np.lexsort(b3.idx.T[::-1])
    assert np.array_equal(f3.idx[o], b3.idx[p])
    assert np.allclose(f3.val[o], b3.val[p], rtol=1e-12, atol=1e-15)
    o = np.lexsort(f2.idx.T[::-1])
    p = np.lexsort(b2.idx.T[::-1])
    assert np.array_equal(f2.idx[o], b2.idx[p]) and np.allclose(f2.val[o], b2.val[p], rtol=1e-12, atol=1e-15)


def _role_weights(fa, fb, fc, na, nb, nc, shape, sig, window):
    """For one unordered triple a <= b <= c (indices), the pair-weight sums each member's
    linewidth receives from all distinct orderings of the other two (written out here by
    hand, in the form a symmetric kernel evaluates them: three deltas shared by the roles)."""
    g = lambda x: O.anharmonic.broadening(x, shape, sig, window)
    d1, d2, d3 = g(fa + fb - fc), g(fa - fb + fc), g(-fa + fb + fc)
    sa = 2 * (1 + nb + nc) * d3 + 2 * (nb - nc) * (d1 - d2)
    sb = 2 * (1 + na + nc) * d2 + 2 * (na - nc) * (d1 - d3)
    sc = 2 * (1 + na + nb) * d1 + 2 * (na - nb) * (d2 - d3)
    return sa, sb, sc


def test_unordered_triple_counting_reproduces_per_mode_sum():
    """gamma from each unordered triple once (roles weighted as above, halved where two
    indices coincide) equals the per-mode ordered-pair sum of Eq. (gamma)."""
    c, f2, f3 = _disordered()
    T, sig, shape, fmin, win = 40.0, 0.3, "lorentz", 0.01, 2.0
    f, E = _solve(c, f2)
    n = f.shape[0]
    F = O.supercell.folded_phi3(f3.idx, f3.val, c.masses)
    V = np.einsum("abc,ai,bj,ck->ijk", F, E, E, E, optimize=True)
    nocc = O.occupation.bose(f, T)
    inv = np.where(f >= fmin, 1.0 / np.where(f > 0, f, 1.0), 0.0)
    K0 = O.anharmonic.prefactor(1) / (2 * np.pi) ** 4
    g = np.zeros(n)
    for a in range(n):
        for b in range(a, n):
            cc = np.arange(b, n)
            sa, sb, sc = _role_weights(f[a], f[b], f[cc], nocc[a], nocc[b], nocc[cc], shape, sig, win)
            K = K0 * V[a, b, cc] ** 2 * inv[a] * inv[b] * inv[cc]
            g[a] += np.sum(K * np.where(cc != b, 1.0, 0.5) * sa)
            if b != a:
                g[b] += np.sum(K * sb)
            g[cc] += np.where(cc != b, K * np.where(a != b, 1.0, 0.5) * sc, 0.0)
    g = np.where(f >= fmin, g, 0.0)
    ref = O.gammapoint.gamma_modes(f3.idx, f3.val, c.masses, f, E, range(n), T, shape, sig, fmin, win)
    assert ref.max() > 0
    assert np.abs(g - ref).max() <= 1e-11 * ref.max()
