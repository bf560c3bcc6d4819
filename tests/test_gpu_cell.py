"""Gamma-only large-cell linewidths (phx_gamma_cell) against the per-mode oracle, with shared
eigenvectors: FP64 to rounding, BF16x3 within the linewidth bar, TF32 reported; ragged tiles,
unsorted modes, both broadenings, the phx_gamma dispatch, and the 1000-atom cell on samples."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

BAR = 1e-4          # gamma relative error on modes with gamma > 1e-3 max (BF16x3)


@pytest.fixture(scope="module")
def phx():
    import paper_2602_23728_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(phx):
    c = phx.Context(0)
    yield c
    c.close()


def _cell(mult, seed, noise=0.05):
    c = P.random_masses(P.fcc_primitive_multiple(5.26, mult), 39.95, 83.8, seed=seed)
    rng = np.random.default_rng(seed)
    c.positions = c.positions + rng.normal(scale=noise, size=c.positions.shape)
    return c


def _setup(ctx, c):
    f2, f3 = P.ifc_lj_vectorised(c, P.LennardJones())
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), np.zeros((1, 3)),
                                    want_vel=False, want_vv=False)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, (1, 1, 1))
    return dict(c=c, f3=f3, h=h, freq=freq[0], evec=evec[0])


def _rel(g, ref):
    big = ref > 1e-3 * ref.max()
    return (np.abs(g - ref)[big] / ref[big]).max()


@pytest.fixture(scope="module")
def c80(ctx):
    return _setup(ctx, _cell((5, 4, 4), 11))       # n = 240: two 128-tiles, ragged tail


@pytest.fixture(scope="module")
def c80_oracle(c80):
    s = c80
    out = {}
    for shape in ("lorentz", "gauss"):
        out[shape] = O.gammapoint.gamma_modes(s["f3"].idx, s["f3"].val, s["c"].masses, s["freq"], s["evec"].real,
                                              range(s["freq"].shape[0]), 40.0, shape, 0.1)
    return out


@pytest.mark.parametrize("shape", ["lorentz", "gauss"])
def test_fp64_matches_oracle(ctx, c80, c80_oracle, shape):
    g = ctx.gamma_cell(c80["h"], c80["freq"], c80["evec"], 40.0, shape=shape, sigma=0.1, precision="fp64")
    ref = c80_oracle[shape]
    assert ref.max() > 0
    assert np.abs(g - ref).max() <= 1e-10 * ref.max()


@pytest.mark.parametrize("prec,tol", [("bf16x3", BAR), ("tf32", 2e-2)])
def test_tensor_core_within_bar(ctx, c80, c80_oracle, prec, tol):
    g = ctx.gamma_cell(c80["h"], c80["freq"], c80["evec"], 40.0, shape="lorentz", sigma=0.1, precision=prec)
    ref = c80_oracle["lorentz"]
    err = _rel(g, ref)
    print(f"{prec}: max rel err {err:.3e}")
    assert err < tol
    assert np.all(g >= -1e-6 * ref.max())


def test_unsorted_modes_give_permuted_result(ctx, c80, c80_oracle):
    perm = np.random.default_rng(5).permutation(c80["freq"].shape[0])
    g = ctx.gamma_cell(c80["h"], c80["freq"][perm], np.ascontiguousarray(c80["evec"][:, perm]), 40.0,
                       shape="lorentz", sigma=0.1, precision="fp64")
    ref = c80_oracle["lorentz"][perm]
    assert np.abs(g - ref).max() <= 1e-10 * ref.max()


def test_gamma_dispatch_equals_cell_entry(ctx, c80):
    a = ctx.gamma(c80["h"], c80["freq"][None], c80["evec"][None], np.array([0], np.int32), 40.0, shape="lorentz",
                  sigma=0.1, precision="bf16x3")[0]
    b = ctx.gamma_cell(c80["h"], c80["freq"], c80["evec"], 40.0, shape="lorentz", sigma=0.1, precision="bf16x3")
    assert np.abs(a - b).max() <= 1e-9 * b.max()


def test_single_partial_tile_small_cell(ctx):
    c = _cell((3, 2, 2), 4)
    pot = P.LennardJones()
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    D = O.gammapoint.dynmat(f2.idx, f2.val.reshape(-1, 9), c.masses)
    lam, E = np.linalg.eigh(D)
    f = np.sign(lam) * np.sqrt(np.abs(lam) * O.constants.EV_A2_AMU_TO_PS2) / O.constants.TWO_PI
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, (1, 1, 1))
    ref = O.gammapoint.gamma_modes(f3.idx, f3.val, c.masses, f, E, range(f.shape[0]), 40.0, "lorentz", 0.3)
    for prec, tol in (("fp64", 1e-10), ("bf16x3", BAR)):
        g = ctx.gamma_cell(h, f, E.astype(np.complex128), 40.0, shape="lorentz", sigma=0.3, precision=prec)
        if prec == "fp64":
            assert np.abs(g - ref).max() <= tol * ref.max()
        else:
            assert _rel(g, ref) < tol


def test_rejects_complex_eigenvectors_and_mesh_handles(ctx, phx, c80):
    with pytest.raises(phx.PhxError):
        ctx.gamma_cell(c80["h"], c80["freq"], c80["evec"] * np.exp(0.3j), 40.0, precision="fp64")
    c = P.fcc_primitive()
    pot = P.LennardJones()
    f3 = P.ifc3_lj(c, pot)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, (2, 2, 2))
    with pytest.raises(phx.PhxError):
        ctx.gamma_cell(h, np.ones(3), np.eye(3, dtype=np.complex128), 40.0, precision="fp64")


@pytest.mark.slow
def test_thousand_atom_cell_sampled_modes(ctx):
    w = P.gamma_disordered_1000()
    s = _setup(ctx, w.crystal)
    kw = dict(shape="lorentz", sigma=w.sigma_thz)
    g16 = ctx.gamma_cell(s["h"], s["freq"], s["evec"], w.temperature, precision="bf16x3", **kw)
    g64 = ctx.gamma_cell(s["h"], s["freq"], s["evec"], w.temperature, precision="fp64", **kw)
    assert g64.max() > 0
    assert _rel(g16, g64) < BAR
    rng = np.random.default_rng(0)
    live = np.nonzero(s["freq"] >= 0.01)[0]
    modes = np.sort(rng.choice(live, 16, replace=False))
    ref = O.gammapoint.gamma_modes(s["f3"].idx, s["f3"].val, w.crystal.masses, s["freq"], s["evec"].real, modes,
                                   w.temperature, "lorentz", w.sigma_thz)
    assert np.abs(g64[modes] - ref).max() <= 1e-9 * g64.max()
    big = ref > 1e-3 * g64.max()
    assert (np.abs(g16[modes] - ref)[big] / ref[big]).max() < BAR
