"""Exchange-pair evaluation (context option 'pair'): one contraction per unordered partner pair
{q', q'' = -(q + q')} with the weights of both orderings, against the plain sum over every q'
(option off) on the same inputs.  Covered: linewidths and WP2, the multi-temperature pass and
the iterative BTE's Gamma1 rows, in both contraction kernels, on odd and even meshes (pairs with
q' = q'' exist only on even ones).  Paper Sec. "Three-Phonon Scattering", Eqs. (phi3_proj),
(gamma), (broadening); Sec. "Boltzmann Transport Equation", Eq. (gamma1).  Both sides run in
BF16x3 on the same operands; the second ordering's |V3|^2 comes from the other contraction
order (q' first instead of q'' first), so they differ by BF16x3 rounding (a few 1e-6 on gamma)
as well as FP32 accumulation order.  Bars: gamma and WP2 2e-5; Gamma1 rows and kappa at the
parity bars against the oracle (row l1 / Gamma0 1e-4, kappa 1e-5).  The oracle comparisons of
the other test files run with the option at its default (on)."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def phx():
    import paper_2602_23728_gb300 as m
    return m


@pytest.fixture()
def ctx(phx):
    c = phx.Context(0)
    yield c
    c.close()


def _rel(a, b):
    big = np.abs(b) > 1e-3 * np.abs(b).max()
    return float((np.abs(a - b)[big] / np.abs(b)[big]).max())


CELLS = {
    # (crystal, mesh, T, sigma); even dimensions give q' = q'' pairs for some q
    "two_atom-345": (lambda: P.random_masses(P.fcc_primitive_multiple(5.26, (2, 1, 1)), 39.95, 83.8, seed=1),
                     (3, 4, 5), 45.0, 0.15),
    "four_atom-332": (lambda: P.random_masses(P.fcc_primitive_multiple(5.26, (2, 2, 1)), 39.95, 83.8, seed=4),
                      (3, 3, 2), 40.0, 0.15),
    "fcc32-222": (lambda: P.fcc_massdisorder_32().crystal, (2, 2, 2), 50.0, 0.1),
    "cell72-333": (lambda: P.random_masses(P.fcc_primitive_multiple(5.26, (4, 3, 2)), 39.95, 83.8, seed=7),
                   (3, 3, 1), 60.0, 0.2),
}


def _setup(ctx, phx, kind):
    make, mesh, T, sig = CELLS[kind]
    c = make()
    f2, f3 = P.ifc_lj_vectorised(c, P.LennardJones())
    q = O.grid.mesh_qred(mesh)
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, want_vel=False,
                                    want_vv=False)
    irr, _, _ = phx.irreducible(mesh, P.identity_rotation())
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    return dict(mesh=mesh, T=T, sig=sig, freq=freq, evec=evec, irr=irr, h=h)


@pytest.mark.parametrize("chain", [1, 2])
@pytest.mark.parametrize("kind", sorted(CELLS))
def test_pair_equals_full_sum(ctx, phx, kind, chain):
    s = _setup(ctx, phx, kind)
    ctx.set_option("chain", chain)
    out = {}
    for pair in (0, 1):
        ctx.set_option("pair", pair)
        out[pair] = ctx.gamma(s["h"], s["freq"], s["evec"], s["irr"], s["T"], "gauss", s["sig"], precision="bf16x3",
                              want_wp2=True)
    dg, dw = _rel(out[1][0], out[0][0]), _rel(out[1][1], out[0][1])
    print(f"{kind} chain={chain}: pair vs full gamma {dg:.2e}, WP2 {dw:.2e}")
    assert out[0][0].max() > 0
    assert dg < 2e-5 and dw < 2e-5


@pytest.mark.parametrize("chain", [1, 2])
def test_pair_multi_t(ctx, phx, chain):
    s = _setup(ctx, phx, "four_atom-332")
    ctx.set_option("chain", chain)
    temps = [20.0, 45.0, 80.0]
    out = {}
    for pair in (0, 1):
        ctx.set_option("pair", pair)
        out[pair] = ctx.gamma_multi_t(s["h"], s["freq"], s["evec"], s["irr"], temps, "lorentz", 0.2,
                                      precision="bf16x3")
    d = max(_rel(out[1][t], out[0][t]) for t in range(len(temps)))
    print(f"multi-T chain={chain}: pair vs full {d:.2e}")
    assert d < 2e-5


def _tr_gauged(c, f2, mesh):
    q = O.grid.mesh_qred(mesh)
    freq, evec, vel = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    irr, pos, sign = O.bte.time_reversal_set(mesh)
    for p in range(q.shape[0]):
        if sign[p] == -1:
            r = irr[pos[p]]
            freq[p], evec[p], vel[p] = freq[r], evec[r].conj(), -vel[r]
    return freq, evec, vel


@pytest.mark.parametrize("chain", [1, 2])
@pytest.mark.parametrize("mesh,shape,sigma", [((3, 3, 3), "gauss", 0.3), ((4, 2, 2), "lorentz", 0.4)])
def test_pair_scattering_rows(ctx, chain, mesh, shape, sigma):
    """Gamma1 rows: an exchange pair adds its summed weight to the columns of both partners."""
    c = P.random_masses(P.fcc_primitive_multiple(5.26, (2, 1, 1)), 39.95, 83.8, seed=1)
    f2, f3 = P.ifc_lj_vectorised(c, P.LennardJones())
    freq, evec, vel = _tr_gauged(c, f2, mesh)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    ctx.set_option("chain", chain)
    out = {}
    for pair in (0, 1):
        ctx.set_option("pair", pair)
        out[pair] = ctx.kappa_sc(c.lattice, c.masses, h, freq, evec, vel, 50.0, shape=shape, sigma=sigma,
                                 precision="bf16x3", max_iter=4, tol=0.0, want_gamma1=True)
    g0, g1 = out[0]["gamma0"], out[0]["gamma1"]
    row_l1 = np.abs(out[1]["gamma1"] - g1).sum(axis=1) / np.maximum(g0.ravel(), 1e-300)
    live = g0.ravel() > 1e-3 * g0.max()
    dk = float(np.abs(out[1]["kappa"] - out[0]["kappa"]).max() / np.abs(out[0]["kappa"]).max())
    print(f"{mesh} {shape} chain={chain}: Gamma0 {_rel(out[1]['gamma0'], g0):.2e}, "
          f"Gamma1 row l1 / Gamma0 {row_l1[live].max():.2e}, kappa {dk:.2e}")
    assert np.abs(g1).max() > 0
    assert _rel(out[1]["gamma0"], g0) < 2e-5
    assert row_l1[live].max() < 1e-4
    assert dk < 1e-5


def test_pair_option_range(ctx, phx):
    with pytest.raises(phx.PhxError):
        ctx.set_option("pair", 2)


@pytest.mark.parametrize("chain", [1, 2])
@pytest.mark.parametrize("kind", ["fcc32-222", "cell72-333"])
def test_side_stream_equals_one_stream(ctx, phx, kind, chain):
    """The fold and Fourier GEMM on a side stream next to the contractions (the chained kernel
    or the two GEMMs; two M buffers, event-ordered) give the one-stream result; only the CTA
    split of the items and so the order of the FP64 accumulation changes."""
    s = _setup(ctx, phx, kind)
    ctx.set_option("chain", chain)
    out = {}
    for side in (0, -1, 16):
        ctx.set_option("side_sms", side)
        if side == 0:
            assert ctx.get_option("side_sms") == 0
        elif side == 16:
            assert ctx.get_option("side_sms") == 16
        else:
            assert ctx.get_option("side_sms") > 0       # the library's default on a full GB300
        out[side] = ctx.gamma(s["h"], s["freq"], s["evec"], s["irr"], s["T"], "gauss", s["sig"],
                              precision="bf16x3")
    for side in (-1, 16):
        d = _rel(out[side], out[0])
        print(f"{kind} chain={chain}: side {side} vs one stream {d:.2e}")
        assert d < 1e-12
