"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only builds inputs: Lennard-Jones crystals, their analytic second- and
third-order interatomic force constants (IFCs), integer symmetry operations and
q-meshes.  It holds none of the scattering method's arithmetic (no dynamical matrix,
eigenvectors, V3, linewidths or conductivity); the oracle and the CUDA library each
implement that on their own.

Units: Angstrom, eV, amu.  IFC2 in eV/A^2, IFC3 in eV/A^3.

The IFCs follow from a pair potential f(r) truncated at r_c (no energy shift, since a
shift changes no derivative).  For a pair with separation vector r = x_j - x_i,
rho = |r|, n = r/rho the Cartesian derivative tensors of f(|r|) are

    H_ab  = (f'' - f'/rho) n_a n_b + (f'/rho) d_ab
    T_abc = (f''' - 3 f''/rho + 3 f'/rho^2) n_a n_b n_c
            + (f''/rho - f'/rho^2) (d_ab n_c + d_ac n_b + d_bc n_a)

and each derivative with respect to x_i instead of x_j flips the sign.  Neighbours are
enumerated over lattice vectors R_l within r_c (the infinite-crystal IFCs), which makes
the acoustic sum rule exact: Phi2(i,i) = sum_j H(r_ij), Phi3(i,i,i) = -sum_j T(r_ij).
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import List, Sequence, Tuple

import numpy as np

# ----------------------------------------------------------------------------- potential


@dataclasses.dataclass(frozen=True)
class LennardJones:
    eps: float = 0.0104     # eV
    sigma: float = 3.4      # Angstrom
    rc: float = 8.5         # Angstrom, plain truncation

    def derivs(self, r):
        """f, f', f'', f''' of 4 eps [(s/r)^12 - (s/r)^6] at r (array)."""
        r = np.asarray(r, dtype=np.float64)
        s6 = (self.sigma / r) ** 6
        s12 = s6 * s6
        e4 = 4.0 * self.eps
        f0 = e4 * (s12 - s6)
        f1 = e4 * (-12.0 * s12 + 6.0 * s6) / r
        f2 = e4 * (156.0 * s12 - 42.0 * s6) / r ** 2
        f3 = e4 * (-2184.0 * s12 + 336.0 * s6) / r ** 3
        return f0, f1, f2, f3


# ----------------------------------------------------------------------------- crystals


@dataclasses.dataclass
class Crystal:
    lattice: np.ndarray      # (3,3) rows are the lattice vectors a1, a2, a3 (Angstrom)
    positions: np.ndarray    # (N,3) Cartesian (Angstrom)
    masses: np.ndarray       # (N,) amu
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def n_modes(self) -> int:
        return 3 * self.n_atoms

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


def fcc_primitive(a: float = 5.26, mass: float = 39.95) -> Crystal:
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    return Crystal(lat, np.zeros((1, 3)), np.array([mass]), "fcc-primitive")


def fcc_conventional(a: float = 5.26, mass: float = 39.95, reps=(1, 1, 1)) -> Crystal:
    """Cubic fcc cell (4 atoms) repeated reps times: 4*prod(reps) atoms."""
    basis = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]]) * a
    pos = []
    for i, j, k in itertools.product(range(reps[0]), range(reps[1]), range(reps[2])):
        pos.append(basis + a * np.array([i, j, k], dtype=np.float64))
    pos = np.concatenate(pos, axis=0)
    lat = np.diag([a * reps[0], a * reps[1], a * reps[2]]).astype(np.float64)
    return Crystal(lat, pos, np.full(pos.shape[0], mass), f"fcc-conv-{reps}")


def fcc_primitive_multiple(a: float, mult: Sequence[int], mass: float = 39.95) -> Crystal:
    """n1 x n2 x n3 multiple of the primitive fcc cell used as a unit cell."""
    prim = fcc_primitive(a, mass)
    n1, n2, n3 = mult
    lat = prim.lattice * np.array([[n1], [n2], [n3]], dtype=np.float64)
    pos = []
    for i, j, k in itertools.product(range(n1), range(n2), range(n3)):
        pos.append(i * prim.lattice[0] + j * prim.lattice[1] + k * prim.lattice[2])
    pos = np.array(pos)
    return Crystal(lat, pos, np.full(pos.shape[0], mass), f"fcc-prim-x{n1}{n2}{n3}")


def supercell(crystal: Crystal, mult: Sequence[int]) -> Crystal:
    """Crystal repeated n1 x n2 x n3 times along its lattice vectors (cell-major ordering)."""
    n1, n2, n3 = mult
    lat = crystal.lattice * np.array([[n1], [n2], [n3]], dtype=np.float64)
    pos, mas = [], []
    for i, j, k in itertools.product(range(n1), range(n2), range(n3)):
        shift = i * crystal.lattice[0] + j * crystal.lattice[1] + k * crystal.lattice[2]
        pos.append(crystal.positions + shift)
        mas.append(crystal.masses)
    return Crystal(lat, np.concatenate(pos), np.concatenate(mas), crystal.name + f"-sc{n1}{n2}{n3}")


def linear_chain(a: float = 4.0, mass: float = 39.95, spacing: float = 20.0) -> Crystal:
    """One atom per cell on a chain along x; the chains are spacing apart in y and z."""
    lat = np.diag([a, spacing, spacing]).astype(np.float64)
    return Crystal(lat, np.zeros((1, 3)), np.array([mass]), "chain")


def random_masses(crystal: Crystal, m1: float, m2: float, seed: int) -> Crystal:
    """50/50 assignment of two masses over the sites: exactly half (rounded down) get m2."""
    rng = np.random.default_rng(seed)
    n = crystal.n_atoms
    m = np.full(n, m1)
    m[rng.permutation(n)[: n // 2]] = m2
    return Crystal(crystal.lattice.copy(), crystal.positions.copy(), m, crystal.name + "-massdis")


# ----------------------------------------------------------------------------- neighbours


def lattice_range(lattice: np.ndarray, rc: float) -> np.ndarray:
    """Integer bounds so that every lattice vector within rc + cell diameter is covered."""
    inv = np.linalg.inv(lattice)
    # |l_i| <= (rc + diam) * |column i of inv(lattice)| bounds the fractional coordinate
    diam = np.linalg.norm(lattice.sum(axis=0)) + np.linalg.norm(lattice, axis=1).sum()
    return np.ceil((rc + diam) * np.linalg.norm(inv, axis=0)).astype(int)


def neighbours(crystal: Crystal, rc: float):
    """All (i, j, R) with 0 < |x_j + R.L - x_i| < rc. Returns i, j, R (int), rvec (Cartesian)."""
    lim = lattice_range(crystal.lattice, rc)
    grid = np.array(list(itertools.product(*[range(-l, l + 1) for l in lim])), dtype=np.int64)
    shifts = grid @ crystal.lattice
    out_i, out_j, out_R, out_r = [], [], [], []
    pos = crystal.positions
    for i in range(crystal.n_atoms):
        d = pos[None, :, :] + shifts[:, None, :] - pos[i][None, None, :]   # (nR, N, 3)
        dist = np.linalg.norm(d, axis=2)
        mask = (dist < rc) & (dist > 1e-8)
        rr, jj = np.nonzero(mask)
        out_i.append(np.full(rr.shape, i))
        out_j.append(jj)
        out_R.append(grid[rr])
        out_r.append(d[rr, jj])
    return (np.concatenate(out_i), np.concatenate(out_j),
            np.concatenate(out_R).astype(np.int64), np.concatenate(out_r))


def _pair_tensors(pot: LennardJones, rvec: np.ndarray):
    rho = np.linalg.norm(rvec, axis=1)
    n = rvec / rho[:, None]
    _, f1, f2, f3 = pot.derivs(rho)
    eye = np.eye(3)
    H = (f2 - f1 / rho)[:, None, None] * n[:, :, None] * n[:, None, :] \
        + (f1 / rho)[:, None, None] * eye[None]
    A = f3 - 3.0 * f2 / rho + 3.0 * f1 / rho ** 2
    B = f2 / rho - f1 / rho ** 2
    nnn = n[:, :, None, None] * n[:, None, :, None] * n[:, None, None, :]
    sym = (eye[None, :, :, None] * n[:, None, None, :]
           + eye[None, :, None, :] * n[:, None, :, None]
           + eye[None, None, :, :] * n[:, :, None, None])
    T = A[:, None, None, None] * nnn + B[:, None, None, None] * sym
    return H, T


@dataclasses.dataclass
class IFC2:
    """Second-order IFC blocks: Phi2(i alpha, (R, j) beta) = val[b, alpha, beta]."""
    idx: np.ndarray    # (nb, 5) int32: i, j, R1, R2, R3
    val: np.ndarray    # (nb, 3, 3) float64

    @property
    def n_blocks(self) -> int:
        return int(self.idx.shape[0])


@dataclasses.dataclass
class IFC3:
    """Third-order IFCs in COO form, home atom a in cell 0.

    Entry k is Phi3(a, (R', b), (R'', c)) with Cartesian components folded into the
    atom index: idx[k] = (3a+alpha, 3b+beta, 3c+gamma, R'1, R'2, R'3, R''1, R''2, R''3).
    """
    idx: np.ndarray    # (nnz, 9) int32
    val: np.ndarray    # (nnz,) float64

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])


def ifc2_lj(crystal: Crystal, pot: LennardJones) -> IFC2:
    ii, jj, RR, rv = neighbours(crystal, pot.rc)
    H, _ = _pair_tensors(pot, rv)
    blocks = {}

    def add(key, m):
        if key in blocks:
            blocks[key] = blocks[key] + m
        else:
            blocks[key] = m.copy()

    for k in range(ii.shape[0]):
        i, j = int(ii[k]), int(jj[k])
        R = tuple(int(x) for x in RR[k])
        add((i, j) + R, -H[k])
        add((i, i, 0, 0, 0), H[k])
    keys = sorted(blocks.keys())
    idx = np.array(keys, dtype=np.int32).reshape(-1, 5)
    val = np.array([blocks[k] for k in keys], dtype=np.float64).reshape(-1, 3, 3)
    return IFC2(idx, val)


def ifc3_lj(crystal: Crystal, pot: LennardJones, drop_rel: float = 1e-15) -> IFC3:
    ii, jj, RR, rv = neighbours(crystal, pot.rc)
    _, T = _pair_tensors(pot, rv)
    acc = {}

    def add(a_atom, b_atom, Rb, c_atom, Rc, t):
        key = (a_atom, b_atom) + tuple(Rb) + (c_atom,) + tuple(Rc)
        if key in acc:
            acc[key] = acc[key] + t
        else:
            acc[key] = t.copy()

    zero = (0, 0, 0)
    for k in range(ii.shape[0]):
        i, j = int(ii[k]), int(jj[k])
        R = tuple(int(x) for x in RR[k])
        t = T[k]
        add(i, i, zero, j, R, t)      # (i, i, j): +T
        add(i, j, R, i, zero, t)      # (i, j, i): +T
        add(i, j, R, j, R, -t)        # (i, j, j): -T
        add(i, i, zero, i, zero, -t)  # (i, i, i): -sum T
    rows, vals = [], []
    vmax = max(float(np.abs(v).max()) for v in acc.values())
    for key, t in sorted(acc.items()):
        a, b = key[0], key[1]
        Rb = key[2:5]
        c = key[5]
        Rc = key[6:9]
        for al, be, ga in itertools.product(range(3), range(3), range(3)):
            v = t[al, be, ga]
            if abs(v) > drop_rel * vmax:
                rows.append((3 * a + al, 3 * b + be, 3 * c + ga) + tuple(Rb) + tuple(Rc))
                vals.append(v)
    return IFC3(np.array(rows, dtype=np.int32).reshape(-1, 9), np.array(vals, dtype=np.float64))


def lj_forces(positions: np.ndarray, lattice: np.ndarray, pot: LennardJones) -> np.ndarray:
    """Forces on the atoms of a periodic cell (all images within rc). Used by the FD pins
    and by the relaxation of the disordered Gamma-only cell."""
    n = positions.shape[0]
    lim = lattice_range(lattice, pot.rc)
    grid = np.array(list(itertools.product(*[range(-l, l + 1) for l in lim])), dtype=np.float64)
    shifts = grid @ lattice
    F = np.zeros_like(positions)
    for i in range(n):
        d = positions[None, :, :] + shifts[:, None, :] - positions[i][None, None, :]
        dist = np.linalg.norm(d, axis=2)
        mask = (dist < pot.rc) & (dist > 1e-8)
        dd = d[mask]
        rr = dist[mask]
        _, f1, _, _ = pot.derivs(rr)
        # E = f(|x_j - x_i|): dE/dx_i = -f' n  ->  F_i = +f' n
        F[i] = (f1[:, None] * dd / rr[:, None]).sum(axis=0)
    return F


# ----------------------------------------------------------------------------- symmetry / mesh


def cubic_rotations_reduced(lattice: np.ndarray) -> np.ndarray:
    """The 48 O_h operations written as integer matrices acting on reduced q coordinates
    (q_red' = A R A^-1 q_red with A the lattice-vector rows).  Only operations that are
    integral in this basis are returned."""
    A = lattice
    Ainv = np.linalg.inv(A)
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3))
            for r, c in enumerate(perm):
                R[r, c] = signs[r]
            # q_cart = B^T q_red with B^T proportional to A^-1; q_red' = A R A^-1 q_red
            M = A @ R @ Ainv
            Mi = np.rint(M)
            if np.abs(M - Mi).max() < 1e-8:
                out.append(Mi.astype(np.int32))
    return np.array(out, dtype=np.int32)


def identity_rotation() -> np.ndarray:
    return np.eye(3, dtype=np.int32)[None]


def mesh_reduced(mesh: Sequence[int]) -> np.ndarray:
    """Gamma-centred mesh points k/n in reduced coordinates, index = (k1*n2 + k2)*n3 + k3."""
    n1, n2, n3 = mesh
    k = np.array(list(itertools.product(range(n1), range(n2), range(n3))), dtype=np.float64)
    return k / np.array([n1, n2, n3], dtype=np.float64)


# ----------------------------------------------------------------------------- workloads


@dataclasses.dataclass
class Workload:
    name: str
    crystal: Crystal
    pot: LennardJones
    mesh: Tuple[int, int, int]
    temperature: float
    sigma_thz: float
    shape: str                 # "gauss" or "lorentz"
    rotations: np.ndarray      # integer reduced rotations used for the irreducible set
    f_min_thz: float = 0.01
    window: float = 2.0

    def ifc2(self) -> IFC2:
        return ifc2_lj(self.crystal, self.pot)

    def ifc3(self) -> IFC3:
        return ifc3_lj(self.crystal, self.pot)


def workload_digest(w: Workload, f2: IFC2, f3: IFC3) -> str:
    """Short SHA-256 over the arrays and scalars that define a workload (IFC entries, masses,
    lattice, mesh, temperature, broadening): a stored result made from these inputs carries
    it, and a reader compares it with the digest of its own inputs before using the result."""
    import hashlib
    h = hashlib.sha256()
    c = w.crystal
    for a in (np.asarray(f2.idx, np.int64), np.asarray(f2.val, np.float64), np.asarray(f3.idx, np.int64),
              np.asarray(f3.val, np.float64), np.asarray(c.masses, np.float64), np.asarray(c.lattice, np.float64),
              np.asarray(w.mesh, np.int64),
              np.asarray([w.temperature, w.sigma_thz, w.window, w.f_min_thz], np.float64)):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(w.shape.encode())
    return h.hexdigest()[:16]


def fcc_monatomic_5() -> Workload:
    """1-atom fcc LJ argon, 5x5x5 mesh, 30 K, Gaussian sigma 0.1 THz, O_h symmetry."""
    c = fcc_primitive()
    return Workload("fcc1-mesh5", c, LennardJones(), (5, 5, 5), 30.0, 0.1, "gauss",
                    cubic_rotations_reduced(c.lattice))


def fcc_massdisorder_32(mesh=(8, 8, 8)) -> Workload:
    """32-atom (2x2x2 conventional) fcc LJ cell, 50/50 masses 39.95/83.8 (seed 2),
    8x8x8 mesh, 50 K, Gaussian sigma 0.1 THz; time reversal only."""
    c = random_masses(fcc_conventional(reps=(2, 2, 2)), 39.95, 83.8, seed=2)
    return Workload("fcc32-massdis-mesh8", c, LennardJones(), tuple(mesh), 50.0, 0.1, "gauss",
                    identity_rotation())


def fcc_conventional_4(mesh=(8, 8, 8), temperature=40.0) -> Workload:
    """4-atom conventional fcc LJ cell with equal masses, O_h symmetry, 40 K."""
    c = fcc_conventional()
    return Workload(f"fcc4-mesh{mesh[0]}", c, LennardJones(), tuple(mesh), temperature, 0.1,
                    "gauss", cubic_rotations_reduced(c.lattice))


def most_cubic_factorisation(n: int) -> Tuple[int, int, int]:
    best = None
    for a in range(1, n + 1):
        if n % a:
            continue
        for b in range(1, n // a + 1):
            if (n // a) % b:
                continue
            c = n // a // b
            key = (max(a, b, c) - min(a, b, c), -min(a, b, c))
            if best is None or key < best[0]:
                best = (key, tuple(sorted((a, b, c), reverse=True)))
    return best[1]


def batched_sweep(n_jobs: int = 64, seed: int = 3) -> List[Workload]:
    """Mass-disordered LJ fcc cells of 1-64 atoms, meshes 4^3..12^3, T in 20-80 K."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n_jobs):
        na = int(rng.integers(1, 65))
        m = int(rng.integers(4, 13))
        T = float(rng.uniform(20.0, 80.0))
        c = fcc_primitive_multiple(5.26, most_cubic_factorisation(na))
        c = random_masses(c, 39.95, 83.8, seed=seed * 1000 + k)
        jobs.append(Workload(f"job{k:02d}-na{na}-mesh{m}", c, LennardJones(), (m, m, m), T,
                             0.1, "gauss", identity_rotation()))
    return jobs


# ----------------------------------------------------------------------------- large Gamma-only cell


def _pairs_within(positions: np.ndarray, lattice: np.ndarray, rc: float):
    """All ordered pairs (i, j, image shift) with 0 < |x_j + R - x_i| < rc (vectorised)."""
    inv = np.linalg.inv(lattice)
    frac = positions @ inv
    span = frac.max(axis=0) - frac.min(axis=0)
    # |frac(x_j + R - x_i)| <= rc |column of inv| bounds R_i within span_i of it
    lim = np.ceil(rc * np.linalg.norm(inv, axis=0) + span).astype(int)
    grid = np.array(list(itertools.product(*[range(-l, l + 1) for l in lim])), dtype=np.int64)
    shifts = grid @ lattice
    I, J, Rk, D = [], [], [], []
    for k, sh in enumerate(shifts):
        d = positions[None, :, :] + sh[None, None, :] - positions[:, None, :]      # (i, j, 3)
        dist2 = (d * d).sum(axis=2)
        ii, jj = np.nonzero((dist2 < rc * rc) & (dist2 > 1e-16))
        I.append(ii); J.append(jj); Rk.append(np.full(ii.shape, k)); D.append(d[ii, jj])
    I = np.concatenate(I); J = np.concatenate(J); Rk = np.concatenate(Rk); D = np.concatenate(D)
    return I, J, grid[Rk], D


def relax_lj(crystal: Crystal, pot: LennardJones, fmax: float = 1e-8, max_steps: int = 20000) -> Crystal:
    """FIRE relaxation of the positions at fixed cell to max |F| < fmax (eV/A)."""
    x = crystal.positions.copy()
    lat = crystal.lattice
    m = crystal.masses[:, None]
    skin = 1.0
    I, J, R, _ = _pairs_within(x, lat, pot.rc + skin)
    x_ref = x.copy()

    def forces(x):
        nonlocal I, J, R, x_ref
        if np.abs(x - x_ref).max() > 0.4 * skin:
            I, J, R, _ = _pairs_within(x, lat, pot.rc + skin)
            x_ref = x.copy()
        d = x[J] + R @ lat - x[I]
        r = np.linalg.norm(d, axis=1)
        ok = r < pot.rc
        _, f1, _, _ = pot.derivs(np.where(ok, r, 1.0))
        fij = np.where(ok, f1 / r, 0.0)[:, None] * d           # force on i from pair (i, j)
        return np.stack([np.bincount(I, weights=fij[:, k], minlength=x.shape[0]) for k in range(3)], axis=1)

    v = np.zeros_like(x)
    dt, dt_max, alpha, n_pos = 0.5, 2.0, 0.1, 0       # time unit sqrt(amu A^2 / eV)
    F = forces(x)
    for _ in range(max_steps):
        if np.abs(F).max() < fmax:
            break
        P = (F * v).sum()
        if P > 0:
            vn, fn = np.linalg.norm(v), np.linalg.norm(F)
            v = (1 - alpha) * v + alpha * F / max(fn, 1e-300) * vn
            n_pos += 1
            if n_pos > 5:
                dt = min(dt * 1.1, dt_max)
                alpha *= 0.99
        else:
            v[:] = 0.0
            dt *= 0.5
            alpha = 0.1
            n_pos = 0
        v = v + dt * F / m
        x = x + dt * v
        F = forces(x)
    return Crystal(lat.copy(), x, crystal.masses.copy(), crystal.name + "-relaxed")


def ifc_lj_vectorised(crystal: Crystal, pot: LennardJones, drop_rel: float = 1e-15):
    """IFC2 blocks and IFC3 COO of a (large) cell, vectorised; the same construction as
    ifc2_lj / ifc3_lj (duplicate entries summed)."""
    ii, jj, RR, rv = _pairs_within(crystal.positions, crystal.lattice, pot.rc)
    H, T = _pair_tensors(pot, rv)
    na = crystal.n_atoms
    # ---- IFC2: (i, j, R) -> -H ; (i, i, 0) -> sum H
    keys2 = np.concatenate([np.stack([ii, jj, RR[:, 0], RR[:, 1], RR[:, 2]], 1),
                            np.stack([ii, ii, 0 * ii, 0 * ii, 0 * ii], 1)])
    vals2 = np.concatenate([-H, H])
    u2, inv2 = np.unique(keys2, axis=0, return_inverse=True)
    acc2 = np.zeros((u2.shape[0], 3, 3))
    np.add.at(acc2, inv2.ravel(), vals2)
    ifc2 = IFC2(u2.astype(np.int32), acc2)
    # ---- IFC3 blocks: (i,i,j)+T, (i,j,i)+T, (i,j,j)-T, (i,i,i)-T ; key (a, b, Rb, c, Rc)
    z = np.zeros_like(RR)
    blocks_k = np.concatenate([
        np.concatenate([ii[:, None], ii[:, None], z, jj[:, None], RR], 1),
        np.concatenate([ii[:, None], jj[:, None], RR, ii[:, None], z], 1),
        np.concatenate([ii[:, None], jj[:, None], RR, jj[:, None], RR], 1),
        np.concatenate([ii[:, None], ii[:, None], z, ii[:, None], z], 1)])
    blocks_v = np.concatenate([T, T, -T, -T])
    u3, inv3 = np.unique(blocks_k, axis=0, return_inverse=True)
    acc3 = np.zeros((u3.shape[0], 3, 3, 3))
    np.add.at(acc3, inv3.ravel(), blocks_v)
    vmax = np.abs(acc3).max()
    a = u3[:, 0]; b = u3[:, 1]; Rb = u3[:, 2:5]; c = u3[:, 5]; Rc = u3[:, 6:9]
    al, be, ga = np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij")
    al, be, ga = al.ravel(), be.ravel(), ga.ravel()
    vals = acc3.reshape(-1, 27)
    keep = np.abs(vals) > drop_rel * vmax
    blk, comp = np.nonzero(keep)
    idx = np.stack([3 * a[blk] + al[comp], 3 * b[blk] + be[comp], 3 * c[blk] + ga[comp],
                    Rb[blk, 0], Rb[blk, 1], Rb[blk, 2], Rc[blk, 0], Rc[blk, 1], Rc[blk, 2]], 1)
    ifc3 = IFC3(idx.astype(np.int32), vals[blk, comp].astype(np.float64))
    return ifc2, ifc3


def gamma_disordered_1000(reps=(10, 10, 10), noise=0.05, seed=5, relax=True):
    """Gamma-only disordered cell: reps x primitive fcc (1000 atoms for 10^3), Gaussian
    positional noise (seeded) relaxed back to the LJ force minimum, 50/50 masses 39.95/83.8;
    Lorentzian smearing (half width 0.05 THz, i.e. sigma = 0.1 THz in the broadening formula)."""
    rng = np.random.default_rng(seed)
    c = fcc_primitive_multiple(5.26, reps)
    c = random_masses(c, 39.95, 83.8, seed=seed)
    c.positions = c.positions + rng.normal(scale=noise, size=c.positions.shape)
    pot = LennardJones()
    if relax:
        c = relax_lj(c, pot)
    return Workload(f"gamma-disordered-{c.n_atoms}", c, pot, (1, 1, 1), 300.0, 0.1, "lorentz",
                    identity_rotation())
