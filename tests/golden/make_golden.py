"""Writes the stored expected values under tests/golden/ by calling only the FP64 oracle
(and the seeded input generators).  Nothing here touches the CUDA library.

    python tests/golden/make_golden.py

fcc32_mesh8_gamma.txt: linewidths of two seeded irreducible q-points of the 32-atom
mass-disordered LJ fcc cell on the 8x8x8 mesh at 50 K (Gaussian sigma 0.1 THz), following
the linewidth equation of the paper's Sec. "Three-Phonon Scattering" (Eqs. gamma,
phi3_proj, broadening) with the readings stated in oracle/anharmonic.py.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O          # noqa: E402
import phx_inputs as P      # noqa: E402


def fcc32_sample_q(n=2, seed=8):
    w = P.fcc_massdisorder_32()
    irr, _, _ = O.grid.irreducible(w.mesh, w.rotations)
    rng = np.random.default_rng(seed)
    return w, np.sort(rng.choice(irr[1:], size=n, replace=False))


def main():
    w, qs = fcc32_sample_q()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    g, wp2 = O.anharmonic.gamma(fc3, w.mesh, freq, evec, qs, w.temperature, w.shape, w.sigma_thz,
                                want_wp2=True)
    path = os.path.join(HERE, "fcc32_mesh8_gamma.txt")
    with open(path, "w") as fh:
        fh.write("# Oracle linewidths (1/ps) and weighted two-phonon phase space (ps^4):\n")
        fh.write("# 32-atom LJ fcc (2x2x2 conventional, a=5.26 A, eps=0.0104 eV, sigma=3.4 A, rc=8.5 A),\n")
        fh.write("# 50/50 masses 39.95/83.8 (seed 2), mesh 8x8x8, T=50 K, Gaussian 0.1 THz, window 2, f_min 0.01.\n")
        fh.write("# Paper Sec. 'Three-Phonon Scattering', Eqs. (gamma), (phi3_proj), (broadening); written by\n")
        fh.write("# tests/golden/make_golden.py from oracle/ only.\n")
        fh.write("# columns: iq nu freq_thz gamma wp2\n")
        for s, iq in enumerate(qs):
            for nu in range(freq.shape[1]):
                fh.write(f"{iq} {nu} {freq[iq, nu]:.17e} {g[s, nu]:.17e} {wp2[s, nu]:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
