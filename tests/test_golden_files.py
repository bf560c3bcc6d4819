"""The stored oracle results under tests/golden/ still describe the inputs the generators
make today (digest of the IFC arrays, masses, lattice, mesh, temperature and broadening),
and hold physically admissible values (linewidths >= 0, a symmetric conductivity with
positive diagonal, cubic-cell isotropy within the mass disorder)."""
import os

import numpy as np

import oracle as O
import phx_inputs as P

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_kappa_file(path):
    digest, kappa = None, None
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("# inputs "):
                digest = line.split()[2]
            elif line.startswith("kappa "):
                kappa = np.array([float(x) for x in line.split()[1:]]).reshape(3, 3)
            elif not line.startswith("#") and line.strip():
                rows.append([float(x) for x in line.split()])
    return digest, kappa, np.array(rows)


def test_fcc32_kappa_file_matches_inputs_and_is_admissible():
    w = P.fcc_massdisorder_32()
    digest, kappa, rows = read_kappa_file(os.path.join(HERE, "fcc32_mesh8_kappa.txt"))
    assert digest == P.workload_digest(w, w.ifc2(), w.ifc3())
    irr, _, _ = O.grid.irreducible(w.mesh, w.rotations)
    assert rows.shape == (len(irr) * 96, 3)
    assert np.array_equal(np.unique(rows[:, 0]).astype(int), np.sort(irr))
    assert np.all(np.isfinite(rows[:, 2])) and rows[:, 2].min() >= 0.0
    assert np.allclose(kappa, kappa.T, rtol=0, atol=1e-14)
    d = np.diag(kappa)
    assert d.min() > 0 and (d.max() - d.min()) / d.mean() < 0.1
    assert np.abs(kappa - np.diag(d)).max() < 0.05 * d.mean()


def test_fcc32_kappa_file_agrees_with_sampled_gamma_file():
    """The two stored files were written by separate oracle runs: their common q-points agree."""
    _, _, rows = read_kappa_file(os.path.join(HERE, "fcc32_mesh8_kappa.txt"))
    g = np.loadtxt(os.path.join(HERE, "fcc32_mesh8_gamma.txt"))
    for iq in np.unique(g[:, 0]).astype(int):
        a = g[g[:, 0] == iq][:, 3]
        freq = g[g[:, 0] == iq][:, 2]
        a = O.anharmonic.degenerate_average(freq, a)
        b = rows[rows[:, 0] == iq][:, 2]
        assert np.abs(a - b).max() <= 1e-10 * a.max()
