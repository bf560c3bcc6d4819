"""q-mesh bookkeeping (paper Sec. "Three-Phonon Scattering": momentum conservation modulo
a reciprocal lattice vector; Sec. "Overview of New Capabilities": scattering restricted to
the irreducible wedge and mapped back to the full grid).

A Gamma-centred n1 x n2 x n3 mesh holds q = (k1/n1, k2/n2, k3/n3) in reduced coordinates,
flat index (k1*n2 + k2)*n3 + k3.
"""
import itertools

import numpy as np


def mesh_int(mesh):
    n1, n2, n3 = mesh
    return np.array(list(itertools.product(range(n1), range(n2), range(n3))), dtype=np.int64)


def mesh_index(k, mesh):
    k = np.mod(np.asarray(k, dtype=np.int64), np.asarray(mesh))
    return (k[..., 0] * mesh[1] + k[..., 1]) * mesh[2] + k[..., 2]


def mesh_qred(mesh):
    return mesh_int(mesh) / np.asarray(mesh, dtype=np.float64)


def third_index(iq, iqp, mesh):
    """Index of q'' = -(q + q') folded back into the mesh (q + q' + q'' = G)."""
    k = mesh_int(mesh)
    return mesh_index(-(k[iq] + k[iqp]), mesh)


def irreducible(mesh, rotations):
    """Orbits of the mesh under the given integer reduced-coordinate rotations together with
    time reversal (q -> -q), which the scattering rates always respect.

    Returns (irr, full_to_irr, weights): irr = sorted representative indices (the smallest
    index of each orbit), full_to_irr[i] = position in irr of the orbit holding i,
    weights = orbit sizes.
    """
    k = mesh_int(mesh)
    nq = k.shape[0]
    ops = [np.asarray(r, dtype=np.int64) for r in rotations]
    ops = ops + [-r for r in ops]
    rep = np.full(nq, -1, dtype=np.int64)
    for i in range(nq):
        if rep[i] >= 0:
            continue
        orbit = {int(mesh_index(r @ k[i], mesh)) for r in ops}
        orbit.add(i)
        m = min(orbit)
        for j in orbit:
            rep[j] = m
    irr = np.unique(rep)
    pos = {int(v): p for p, v in enumerate(irr)}
    full_to_irr = np.array([pos[int(r)] for r in rep], dtype=np.int64)
    weights = np.bincount(full_to_irr, minlength=irr.shape[0])
    return irr, full_to_irr, weights
