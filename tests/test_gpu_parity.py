"""GPU parity: the CUDA library through its C ABI against the FP64 oracle, element by
element on the same seeded inputs.  Tolerances: FP64 path 1e-10 relative (summation order
only); per-mode comparisons use the same eigenvectors on both sides."""
import os

import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def phx():
    import paper_2602_23728_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(phx):
    c = phx.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def fcc1(ctx):
    w = P.fcc_monatomic_5()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, vel, vv = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
    return dict(w=w, f2=f2, f3=f3, q=q, freq=freq, evec=evec, vel=vel, vv=vv,
                fc3=O.anharmonic.FC3(f3.idx, f3.val, c.masses))


def _rel(a, b, mask=None):
    a = np.asarray(a); b = np.asarray(b)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# ----------------------------------------------------------------------------- harmonic

def _check_harmonic(w, f2, q, freq, evec, vel, vv):
    c = w.crystal
    fo, eo, vo = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    # compare eigenvalues (f|f|): near f = 0 the frequency is the root of rounding noise
    fmax = np.abs(fo).max()
    assert np.abs(freq * np.abs(freq) - fo * np.abs(fo)).max() < 1e-11 * fmax ** 2
    n = freq.shape[1]
    for k in range(q.shape[0]):
        D = O.harmonic.dynamical_matrix(f2.idx, f2.val, c.masses, q[k])
        lam = np.sign(freq[k]) * (2 * np.pi * freq[k]) ** 2 / O.constants.EV_A2_AMU_TO_PS2
        res = D @ evec[k] - evec[k] * lam[None, :]
        scale = (2 * np.pi * fmax) ** 2 / O.constants.EV_A2_AMU_TO_PS2     # largest eigenvalue
        assert np.abs(res).max() < 1e-11 * scale
        assert np.abs(evec[k].conj().T @ evec[k] - np.eye(n)).max() < 1e-12
        # gauge: a largest-modulus component of every column is real and positive (components
        # whose moduli tie to rounding may be picked in either order)
        mod2 = np.abs(evec[k]) ** 2
        near = mod2 >= mod2.max(axis=0, keepdims=True) * (1 - 1e-12)
        pos = (evec[k].real > 0) & (np.abs(evec[k].imag) < 1e-14)
        assert np.all((near & pos).any(axis=0))
        ok = freq[k] > 0.01
        if not ok.any():
            continue
        # velocities with the GPU eigenvectors on both sides (per-mode values are basis dependent)
        v_or = O.harmonic.velocities(f2.idx, f2.val, c.masses, c.lattice, q[k], freq[k], evec[k])
        assert np.abs(vel[k][ok] - v_or[ok]).max() < 1e-9 * max(1.0, np.abs(v_or).max())
        # invariant products against the oracle's own eigenvectors (basis independent)
        vv_or = O.harmonic.velocity_products(f2.idx, f2.val, c.masses, c.lattice, q[k], fo[k], eo[k])
        assert np.abs(vv[k][ok] - vv_or[ok]).max() < 1e-8 * max(1.0, np.abs(vv_or).max())


def test_harmonic_fcc1(fcc1):
    _check_harmonic(fcc1["w"], fcc1["f2"], fcc1["q"], fcc1["freq"], fcc1["evec"], fcc1["vel"], fcc1["vv"])


def test_harmonic_fcc32_subset(ctx):
    w = P.fcc_massdisorder_32()
    f2 = w.ifc2()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)[np.r_[0:3, 100:103, 257, 511]]
    freq, evec, vel, vv = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
    _check_harmonic(w, f2, q, freq, evec, vel, vv)


def test_harmonic_ragged_two_atom(ctx):
    c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
    c = P.Crystal(c.lattice, c.positions, np.array([39.95, 83.8]))
    w = P.Workload("two", c, P.LennardJones(), (3, 4, 5), 40.0, 0.1, "gauss", P.identity_rotation())
    f2 = w.ifc2()
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, vel, vv = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
    _check_harmonic(w, f2, q, freq, evec, vel, vv)


def test_velocity_products_fp32_option(ctx):
    """PHX_OPT_VEL_FP32: dD/dq E with FP32 products and sums, FP64 in and out.  Frequencies and
    eigenvectors are unchanged (the eigensolve stays FP64); velocities and the basis-invariant
    velocity products stay within 1e-6 of the FP64 run (relative to their largest entry)."""
    w = P.fcc_massdisorder_32()
    f2 = w.ifc2()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)[np.r_[0:3, 100:103, 257, 511]]
    ref = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
    ctx.set_option("vel_fp32", 1)
    try:
        assert ctx.get_option("vel_fp32") == 1
        got = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
    finally:
        ctx.set_option("vel_fp32", 0)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    for a, b in ((got[2], ref[2]), (got[3], ref[3])):
        d = np.abs(a - b).max() / np.abs(b).max()
        print(f"FP32 velocity products: max rel diff {d:.2e}")
        assert 0 < np.abs(b).max() and d < 1e-6


def test_harmonic_time_reversal_fill(ctx):
    """PHX_OPT_HARMONIC_TR (default on): one q of every {q, -q} pair is solved and the other
    filled by time reversal, D(-q) = conj D(q).  On the full 8x8x8 mesh of the 32-atom cell, and
    on a shuffled list with a repeated point, a point given as -q + G and the self-conjugate
    points: the filled points satisfy the oracle's eigenproblem (residual, unitarity, gauge,
    velocities), e(-q) is exactly conj e(q), and frequencies, velocities and velocity products
    equal the run that solves every q on its own."""
    w = P.fcc_massdisorder_32()
    f2 = w.ifc2()
    c = w.crystal
    qm = O.grid.mesh_qred(w.mesh)
    rng = np.random.default_rng(4)
    sub = rng.permutation(len(qm))[:40]
    extra = np.array([qm[sub[0]], -qm[sub[0]] + np.array([1.0, 2.0, -1.0]), qm[sub[1]], qm[0], [0.5, 0.5, 0.0]])
    for q in (qm, np.concatenate([qm[sub], extra])):
        assert ctx.get_option("harmonic_tr") == 1
        got = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
        ctx.set_option("harmonic_tr", 0)
        try:
            ref = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
        finally:
            ctx.set_option("harmonic_tr", 1)
        fmax = np.abs(ref[0]).max()
        assert np.abs(got[0] * np.abs(got[0]) - ref[0] * np.abs(ref[0])).max() < 1e-11 * fmax ** 2
        # per-mode velocities depend on the basis of a degenerate set: compare them on isolated
        # modes, the basis-invariant products on all
        gap = np.minimum(np.diff(ref[0], axis=1, prepend=-np.inf), np.diff(ref[0], axis=1, append=np.inf))
        ok = ref[0] > 0.01
        iso = ok & (gap > 1e-5 * fmax)
        assert np.abs(got[2][iso] - ref[2][iso]).max() < 1e-8 * np.abs(ref[2]).max()
        assert np.abs(got[3][ok] - ref[3][ok]).max() < 1e-8 * np.abs(ref[3]).max()
        # pairs in the list: the later member is the conjugate (or a copy) of the earlier one
        n_pairs = 0
        for i in range(len(q)):
            for j in range(i):
                d_neg, d_same = q[j] + q[i], q[j] - q[i]
                if np.all(np.abs(d_same - np.rint(d_same)) < 1e-9):
                    assert np.array_equal(got[1][i], got[1][j])
                    n_pairs += 1
                    break
                if np.all(np.abs(d_neg - np.rint(d_neg)) < 1e-9):
                    assert np.array_equal(got[1][i], got[1][j].conj())
                    assert np.array_equal(got[2][i], -got[2][j])
                    n_pairs += 1
                    break
        assert n_pairs >= 3
        # the filled points against the oracle's dynamical matrices
        filled = [i for i in range(len(q)) if any(
            np.all(np.abs((q[j] + q[i]) - np.rint(q[j] + q[i])) < 1e-9) for j in range(i))][:6]
        _check_harmonic(w, f2, q[filled], got[0][filled], got[1][filled], got[2][filled], got[3][filled])


# ----------------------------------------------------------------------------- linewidths, FP64

def test_gamma_fp64_fcc1_all_irreducible(ctx, phx, fcc1):
    w = fcc1["w"]
    c = w.crystal
    irr, _, _ = phx.irreducible(w.mesh, w.rotations)
    h = ctx.fc3(c.lattice, c.masses, fcc1["f3"].idx, fcc1["f3"].val, w.mesh)
    g, wp = ctx.gamma(h, fcc1["freq"], fcc1["evec"], irr, w.temperature, w.shape, w.sigma_thz, want_wp2=True)
    go, wo = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], irr, w.temperature,
                                w.shape, w.sigma_thz, want_wp2=True)
    assert go.max() > 0
    assert _rel(g, go) < 1e-10
    assert _rel(wp, wo) < 1e-10


@pytest.mark.parametrize("shape,window,T,fmin", [("lorentz", 2.0, 30.0, 0.01), ("gauss", 50.0, 80.0, 0.01),
                                                 ("gauss", 2.0, 30.0, 1.0)])
def test_gamma_fp64_variants(ctx, phx, fcc1, shape, window, T, fmin):
    w = fcc1["w"]
    c = w.crystal
    irr = np.array([7, 31, 62], dtype=np.int32)
    h = ctx.fc3(c.lattice, c.masses, fcc1["f3"].idx, fcc1["f3"].val, w.mesh)
    g = ctx.gamma(h, fcc1["freq"], fcc1["evec"], irr, T, shape, 0.1, window=window, f_min=fmin)
    go = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fcc1["freq"], fcc1["evec"], irr, T, shape, 0.1,
                            f_min=fmin, window=window)
    assert _rel(g, go) < 1e-10
    assert np.all(g[fcc1["freq"][irr] < fmin] == 0)


def test_gamma_fp64_ragged_two_atom_mesh345(ctx, phx):
    c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
    c = P.Crystal(c.lattice, c.positions, np.array([39.95, 83.8]))
    mesh = (3, 4, 5)
    pot = P.LennardJones()
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    q = O.grid.mesh_qred(mesh)
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q)
    irr, _, _ = phx.irreducible(mesh, P.identity_rotation())
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    g = ctx.gamma(h, freq, evec, irr, 45.0, "gauss", 0.15)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    go = O.anharmonic.gamma(fc3, mesh, freq, evec, irr, 45.0, "gauss", 0.15)
    assert go.max() > 0
    assert _rel(g, go) < 1e-10


def test_gamma_fp64_fcc32_sampled_vs_golden(ctx, phx):
    """Full 8x8x8 / 96-mode size, two seeded irreducible q, against stored oracle values."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "fcc32_mesh8_gamma.txt"))
    qs = np.unique(rows[:, 0]).astype(np.int32)
    w = P.fcc_massdisorder_32()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, w.mesh)
    assert h.num_d == 27
    g, wp = ctx.gamma(h, freq, evec, qs, w.temperature, w.shape, w.sigma_thz, want_wp2=True)
    ref_g = rows[:, 3].reshape(len(qs), -1)
    ref_w = rows[:, 4].reshape(len(qs), -1)
    assert np.allclose(freq[qs], rows[:, 2].reshape(len(qs), -1), atol=1e-9)
    assert _rel(g, ref_g) < 1e-9
    assert _rel(wp, ref_w) < 1e-9


# ----------------------------------------------------------------------------- transport

def test_unfold_and_kappa_end_to_end_fcc1(ctx, phx, fcc1):
    """GPU harmonic + GPU gamma + unfold + kappa against the oracle chain with its own
    eigenvectors; degenerate-averaged gamma and invariant v(x)v make it basis independent."""
    w = fcc1["w"]
    c = w.crystal
    irr, f2i, _ = phx.irreducible(w.mesh, w.rotations)
    h = ctx.fc3(c.lattice, c.masses, fcc1["f3"].idx, fcc1["f3"].val, w.mesh)
    g = ctx.gamma(h, fcc1["freq"], fcc1["evec"], irr, w.temperature, w.shape, w.sigma_thz)
    gf = ctx.unfold(fcc1["freq"], irr, g, f2i)
    K = ctx.kappa_rta(c.lattice, c.masses, fcc1["freq"], gf, w.temperature, vv=fcc1["vv"])
    f2 = fcc1["f2"]
    fo, eo, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, fcc1["q"])
    go = O.anharmonic.gamma(fcc1["fc3"], w.mesh, fo, eo, irr, w.temperature, w.shape, w.sigma_thz)
    go = np.array([O.anharmonic.degenerate_average(fo[i], go[s]) for s, i in enumerate(irr)])
    gfo = O.transport.unfold(go, f2i)
    assert _rel(gf, gfo) < 1e-9
    vvo = np.array([O.harmonic.velocity_products(f2.idx, f2.val, c.masses, c.lattice, fcc1["q"][k], fo[k], eo[k])
                    for k in range(fo.shape[0])])
    Ko = O.transport.kappa_rta_vv(fo, vvo, gfo, w.temperature, c.volume)
    assert np.linalg.norm(K - Ko) / np.linalg.norm(Ko) < 1e-9
    # per-mode velocity form as well, with the GPU eigenvectors
    Kv = ctx.kappa_rta(c.lattice, c.masses, fcc1["freq"], gf, w.temperature, vel=fcc1["vel"])
    Kvo = O.transport.kappa_rta(fcc1["freq"], fcc1["vel"], gf, w.temperature, c.volume)
    assert np.linalg.norm(Kv - Kvo) / np.linalg.norm(Kvo) < 1e-12


# ----------------------------------------------------------------------------- memory paths, errors

def test_device_memory_path_matches_host(ctx, phx, fcc1):
    import torch
    w = fcc1["w"]
    c = w.crystal
    irr, _, _ = phx.irreducible(w.mesh, w.rotations)
    h = ctx.fc3(c.lattice, c.masses, fcc1["f3"].idx, fcc1["f3"].val, w.mesh)
    g_host = ctx.gamma(h, fcc1["freq"], fcc1["evec"], irr, w.temperature, w.shape, w.sigma_thz)
    dev = torch.device("cuda:0")
    f_d = torch.from_numpy(fcc1["freq"]).to(dev)
    e_d = torch.from_numpy(fcc1["evec"]).to(dev)
    i_d = torch.from_numpy(np.asarray(irr, np.int32)).to(dev)
    g_d = torch.zeros((len(irr), 3), dtype=torch.float64, device=dev)
    ctx.gamma(h, f_d, e_d, i_d, w.temperature, w.shape, w.sigma_thz, gamma=g_d)
    torch.cuda.synchronize()
    # same kernels; only the order of the floating-point atomics may differ between runs
    assert _rel(g_d.cpu().numpy(), g_host) < 1e-13
    q_d = torch.from_numpy(fcc1["q"]).to(dev)
    fr = torch.zeros((125, 3), dtype=torch.float64, device=dev)
    ev = torch.zeros((125, 3, 3), dtype=torch.complex128, device=dev)
    ctx.harmonic(c.lattice, c.masses, fcc1["f2"].idx, fcc1["f2"].val.reshape(-1, 9), q_d, freq=fr, evec=ev,
                 want_vel=False, want_vv=False)
    torch.cuda.synchronize()
    assert np.array_equal(fr.cpu().numpy(), fcc1["freq"])


def test_invalid_inputs_raise(ctx, phx, fcc1):
    w = fcc1["w"]
    c = w.crystal
    h = ctx.fc3(c.lattice, c.masses, fcc1["f3"].idx, fcc1["f3"].val, w.mesh)
    with pytest.raises(phx.PhxError):
        ctx.gamma(h, fcc1["freq"], fcc1["evec"], np.array([125], np.int32), 30.0)
    with pytest.raises(phx.PhxError):
        ctx.gamma(h, fcc1["freq"], fcc1["evec"], np.array([1], np.int32), -5.0)
    with pytest.raises(phx.PhxError):
        ctx.gamma(h, fcc1["freq"], fcc1["evec"], np.array([1], np.int32), 30.0, sigma=0.0)
    bad = fcc1["f3"].idx.copy()
    bad[0, 1] = 99
    with pytest.raises(phx.PhxError):
        ctx.fc3(c.lattice, c.masses, bad, fcc1["f3"].val, w.mesh)
    # empty request is a no-op
    out = ctx.gamma(h, fcc1["freq"], fcc1["evec"], np.zeros(0, np.int32), 30.0)
    assert out.shape == (0, 3)
    # the context is still usable after the errors
    g = ctx.gamma(h, fcc1["freq"], fcc1["evec"], np.array([3], np.int32), 30.0)
    assert np.isfinite(g).all()
