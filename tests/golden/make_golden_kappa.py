"""Writes tests/golden/fcc32_mesh8_kappa.txt: the FP64 oracle's linewidths of every
irreducible mode and the RTA conductivity of the 32-atom mass-disordered LJ fcc cell on the
8x8x8 mesh (50 K, Gaussian sigma 0.1 THz, window 2, f_min 0.01 THz).  Only oracle/ and the
seeded input generators are called; nothing here touches the CUDA library.

    python tests/golden/make_golden_kappa.py [--workers 7]

Follows the paper's Sec. "Three-Phonon Scattering" (Eqs. gamma, phi3_proj, broadening) for
the linewidths, with linewidths averaged over degenerate sets and the basis-invariant
velocity products in Eq. (rta) (Sec. "Boltzmann Transport Equation").  The irreducible
q-points are split over worker processes (spawned, one BLAS thread each); every q-point's
linewidths are the oracle's own sum over all q' of the mesh.

The header holds phx_inputs.workload_digest of the inputs (IFC arrays, masses, lattice, mesh,
temperature, broadening): a reader compares it with the digest of its own inputs before it
uses the file.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fcc32_mesh8_kappa.txt")

_STATE = {}


def _init(freq, evec, fc3_args, mesh, T, shape, sigma, window, f_min):
    sys.path.insert(0, ROOT)
    import oracle as O
    _STATE.update(O=O, freq=freq, evec=evec, fc3=O.anharmonic.FC3(*fc3_args), mesh=mesh, T=T, shape=shape,
                  sigma=sigma, window=window, f_min=f_min)


def _one(iq):
    s = _STATE
    g = s["O"].anharmonic.gamma(s["fc3"], s["mesh"], s["freq"], s["evec"], [iq], s["T"], s["shape"], s["sigma"],
                                s["f_min"], s["window"])
    return iq, g[0]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"          # inherited by the spawned workers
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    import phx_inputs as P

    w = P.fcc_massdisorder_32()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    irr, f2i, _ = O.grid.irreducible(w.mesh, w.rotations)
    t0 = time.time()
    ctxm = mp.get_context("spawn")
    res = {}
    with ctxm.Pool(args.workers, initializer=_init,
                   initargs=(freq, evec, (f3.idx, f3.val, c.masses), tuple(w.mesh), w.temperature, w.shape,
                             w.sigma_thz, w.window, w.f_min_thz)) as pool:
        for k, (iq, g) in enumerate(pool.imap_unordered(_one, [int(i) for i in irr])):
            res[iq] = g
            print(f"{k + 1}/{len(irr)} q-points, {time.time() - t0:.0f} s", flush=True)
    g_irr = np.array([O.anharmonic.degenerate_average(freq[i], res[int(i)]) for i in irr])
    vv = np.array([O.harmonic.velocity_products(f2.idx, f2.val, c.masses, c.lattice, q[k], freq[k], evec[k])
                   for k in range(q.shape[0])])
    g_full = O.transport.unfold(g_irr, f2i)
    kappa = O.transport.kappa_rta_vv(freq, vv, g_full, w.temperature, c.volume, f_min=w.f_min_thz)
    with open(OUT, "w") as fh:
        fh.write("# Oracle linewidths (1/ps, degenerate-averaged) of every irreducible mode and the RTA\n")
        fh.write("# conductivity (W/(m K), basis-invariant velocity products) of the 32-atom LJ fcc cell\n")
        fh.write("# (2x2x2 conventional, a=5.26 A, eps=0.0104 eV, sigma=3.4 A, rc=8.5 A), 50/50 masses\n")
        fh.write("# 39.95/83.8 (seed 2), mesh 8x8x8 (time reversal: 260 irreducible q), T=50 K, Gaussian\n")
        fh.write("# 0.1 THz, window 2, f_min 0.01 THz.  Paper Sec. 'Three-Phonon Scattering' (Eqs. gamma,\n")
        fh.write("# phi3_proj, broadening) and Sec. 'Boltzmann Transport Equation' (Eq. rta); written by\n")
        fh.write("# tests/golden/make_golden_kappa.py from oracle/ only.\n")
        fh.write(f"# inputs {P.workload_digest(w, f2, f3)}\n")
        fh.write("kappa " + " ".join(f"{x:.17e}" for x in kappa.ravel()) + "\n")
        fh.write("# columns: iq nu gamma\n")
        for s, iq in enumerate(irr):
            for nu in range(freq.shape[1]):
                fh.write(f"{iq} {nu} {g_irr[s, nu]:.15e}\n")
    print("wrote", OUT, "kappa diag", np.diag(kappa), f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
