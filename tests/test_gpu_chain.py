"""Chained eigenvector contractions (one tcgen05 kernel: X kept in tensor memory, stage-3 A
operand read from tensor memory) against the FP64 oracle on the same eigenvectors, and
against the two-GEMM path on the same inputs.

Paper Sec. "Three-Phonon Scattering", Eqs. (phi3_proj), (gamma), (broadening).  Bars as in
test_gpu_tc.py: BF16x3 gamma within 1e-4 on modes above 1e-3 of the maximum, TF32 within
2e-2; the two tensor-core paths differ only in FP32 accumulation order (1e-5)."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
TOL = {"bf16x3": 1e-4, "tf32": 2e-2}


@pytest.fixture(scope="module")
def phx():
    import paper_2602_23728_gb300 as m
    return m


@pytest.fixture()
def ctx(phx):
    c = phx.Context(0)
    yield c
    c.close()


def _err(g, go):
    big = go > 1e-3 * go.max()
    return float((np.abs(g - go)[big] / go[big]).max())


def _cell(kind):
    """(crystal, mesh, T, sigma, irreducible list or None) of the cases: n = 3, 6, 12, 72 modes."""
    if kind == "fcc1":
        w = P.fcc_monatomic_5()
        return w.crystal, w.mesh, w.temperature, w.sigma_thz, w.rotations
    if kind == "two_atom":
        c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
        return P.Crystal(c.lattice, c.positions, np.array([39.95, 83.8])), (3, 4, 5), 45.0, 0.15, None
    if kind == "four_atom":
        c = P.random_masses(P.fcc_primitive_multiple(5.26, (2, 2, 1)), 39.95, 83.8, seed=4)
        return c, (3, 3, 2), 40.0, 0.15, None
    if kind == "cell72":
        c = P.random_masses(P.fcc_primitive_multiple(5.26, (4, 3, 2)), 39.95, 83.8, seed=7)
        return c, (2, 1, 1), 60.0, 0.2, None
    raise ValueError(kind)


def _setup(ctx, phx, kind):
    c, mesh, T, sig, rot = _cell(kind)
    pot = P.LennardJones()
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    q = O.grid.mesh_qred(mesh)
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, want_vel=False,
                                    want_vv=False)
    irr, _, _ = phx.irreducible(mesh, rot if rot is not None else P.identity_rotation())
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    return dict(c=c, mesh=mesh, T=T, sig=sig, freq=freq, evec=evec, irr=irr, h=h, fc3=fc3)


@pytest.mark.parametrize("kind", ["fcc1", "two_atom", "four_atom", "cell72"])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_chain_matches_oracle(ctx, phx, kind, prec):
    s = _setup(ctx, phx, kind)
    ctx.set_option("chain", 1)
    g, wp = ctx.gamma(s["h"], s["freq"], s["evec"], s["irr"], s["T"], "gauss", s["sig"], precision=prec,
                      want_wp2=True)
    go, wo = O.anharmonic.gamma(s["fc3"], s["mesh"], s["freq"], s["evec"], s["irr"], s["T"], "gauss", s["sig"],
                                want_wp2=True)
    print(f"{prec} {kind} ({s['freq'].shape[1]} modes): chained gamma max rel err {_err(g, go):.3e}")
    assert go.max() > 0
    assert _err(g, go) < TOL[prec]
    assert _err(wp, wo) < 1e-5


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_chain_equals_two_gemm_path(ctx, phx, prec):
    """Same arithmetic in both tensor-core paths, different FP32 summation order."""
    s = _setup(ctx, phx, "cell72")
    ctx.set_option("chain", 1)
    g1 = ctx.gamma(s["h"], s["freq"], s["evec"], s["irr"], s["T"], "gauss", s["sig"], precision=prec)
    ctx.set_option("chain", 2)
    g2 = ctx.gamma(s["h"], s["freq"], s["evec"], s["irr"], s["T"], "gauss", s["sig"], precision=prec)
    big = g2 > 1e-3 * g2.max()
    d = float((np.abs(g1 - g2)[big] / g2[big]).max())
    print(f"{prec}: chained vs two-GEMM max rel diff {d:.3e}")
    assert d < (1e-5 if prec == "bf16x3" else 1e-3)


def test_chain_lorentzian_fcc1(ctx, phx):
    s = _setup(ctx, phx, "fcc1")
    ctx.set_option("chain", 1)
    g = ctx.gamma(s["h"], s["freq"], s["evec"], s["irr"], s["T"], "lorentz", 0.1, precision="bf16x3")
    go = O.anharmonic.gamma(s["fc3"], s["mesh"], s["freq"], s["evec"], s["irr"], s["T"], "lorentz", 0.1)
    assert _err(g, go) < 1e-4
