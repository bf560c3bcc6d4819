"""Several temperatures from one contraction (phx_gamma_multi_t) against single-temperature
calls and the oracle at each temperature (the oracle's split is pinned by P10)."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TEMPS = [20.0, 50.0, 120.0, 300.0, 600.0]     # two tensor-core passes (4 + 1)


@pytest.fixture(scope="module")
def setup():
    import paper_2602_23728_gb300 as m
    ctx = m.Context(0)
    c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
    c = P.Crystal(c.lattice, c.positions, np.array([39.95, 83.8]), "fcc2")
    pot = P.LennardJones()
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    mesh = (4, 4, 4)
    q = O.grid.mesh_qred(mesh)
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, want_vel=False,
                                    want_vv=False)
    irr, _, _ = m.irreducible(mesh, P.identity_rotation())
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    yield dict(ctx=ctx, c=c, f3=f3, mesh=mesh, freq=freq, evec=evec, irr=irr.astype(np.int32), h=h)
    ctx.close()


@pytest.mark.parametrize("prec,chain", [("bf16x3", 2), ("tf32", 2), ("fp64", 0), ("bf16x3", 1), ("tf32", 1)])
def test_multi_t_equals_single_calls(setup, prec, chain):
    """chain 1: the chained tensor-core kernel (forced on at 6 modes), 2: the two GEMMs."""
    s = setup
    s["ctx"].set_option("chain", chain)
    try:
        g = s["ctx"].gamma_multi_t(s["h"], s["freq"], s["evec"], s["irr"], TEMPS, precision=prec)
        assert g.shape == (len(TEMPS), len(s["irr"]), s["freq"].shape[1])
        for t, T in enumerate(TEMPS):
            one = s["ctx"].gamma(s["h"], s["freq"], s["evec"], s["irr"], T, precision=prec)
            assert np.abs(g[t] - one).max() <= 1e-5 * one.max()
        assert np.all(np.diff(g.max(axis=(1, 2))) > 0)       # more phonons, faster scattering
    finally:
        s["ctx"].set_option("chain", 0)


@pytest.mark.parametrize("chain", [1, 2])
def test_multi_t_matches_oracle(setup, chain):
    s = setup
    s["ctx"].set_option("chain", chain)
    try:
        g = s["ctx"].gamma_multi_t(s["h"], s["freq"], s["evec"], s["irr"], TEMPS, precision="bf16x3")
    finally:
        s["ctx"].set_option("chain", 0)
    fc3 = O.anharmonic.FC3(s["f3"].idx, s["f3"].val, s["c"].masses)
    sub = [0, 3, 7]
    ref0, v2 = O.anharmonic.gamma(fc3, s["mesh"], s["freq"], s["evec"], s["irr"][sub], TEMPS[0], keep_v2=True)
    for t, T in enumerate(TEMPS):
        ref = ref0 if t == 0 else O.anharmonic.gamma_from_v2(v2, s["mesh"], s["freq"], s["irr"][sub], T)
        big = ref > 1e-3 * ref.max()
        assert (np.abs(g[t][sub] - ref)[big] / ref[big]).max() < 1e-4


def test_multi_t_rejects_bad_temperature(setup):
    import paper_2602_23728_gb300 as m
    s = setup
    with pytest.raises(m.PhxError):
        s["ctx"].gamma_multi_t(s["h"], s["freq"], s["evec"], s["irr"], [50.0, -1.0], precision="bf16x3")
