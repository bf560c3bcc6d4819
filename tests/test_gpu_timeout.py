"""Bounded device waits of the tensor-core kernels: with the load producer told to issue
nothing (no copy and no MMA is ever in flight) and a 1 ms wait limit, the first barrier wait
runs out, the kernel retires, the call returns PHX_ERR_TIMEOUT, and the next normal call on
the same context matches the oracle.  No GPU fault is involved: the kernels give up on
their own and report through the status word."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
PHX_ERR_TIMEOUT = 4


@pytest.fixture(scope="module")
def phx():
    import paper_2602_23728_gb300 as m
    return m


@pytest.mark.parametrize("chain", [1, 2])
def test_starved_producer_times_out_then_context_works(phx, chain):
    w = P.fcc_monatomic_5()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)
    ctx = phx.Context(0)
    try:
        freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, want_vel=False,
                                        want_vv=False)
        irr, _, _ = phx.irreducible(w.mesh, w.rotations)
        h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, w.mesh)
        ctx.set_option("chain", chain)
        ctx.set_option("wait_limit_ns", 1_000_000)
        ctx.set_option("starve", 1)
        with pytest.raises(phx.PhxError) as ei:
            ctx.gamma(h, freq, evec, irr, w.temperature, w.shape, w.sigma_thz, precision="bf16x3")
        assert ei.value.status == PHX_ERR_TIMEOUT
        ctx.set_option("starve", 0)
        ctx.set_option("wait_limit_ns", 2_000_000_000)
        g = ctx.gamma(h, freq, evec, irr, w.temperature, w.shape, w.sigma_thz, precision="bf16x3")
        fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
        go = O.anharmonic.gamma(fc3, w.mesh, freq, evec, irr, w.temperature, w.shape, w.sigma_thz)
        big = go > 1e-3 * go.max()
        assert float((np.abs(g - go)[big] / go[big]).max()) < 1e-4
    finally:
        ctx.close()


def test_option_arguments_checked(phx):
    ctx = phx.Context(0)
    try:
        with pytest.raises(phx.PhxError):
            ctx.set_option("chain", 3)
        with pytest.raises(phx.PhxError):
            ctx.set_option("wait_limit_ns", 10)
    finally:
        ctx.close()
