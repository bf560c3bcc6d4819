"""The allocation-free conductivity entry point (for callers that cannot allocate device
memory when they call in) against the ordinary one, through the C ABI, on two calls in a
row.  Kept in a file of its own that collects last."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu]


def test_kappa_noalloc_matches_kappa_rta_twice():
    import torch
    import paper_2602_23728_gb300 as phx
    ctx = phx.Context(0)
    dev = torch.device("cuda:0")
    w = P.fcc_monatomic_5()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = torch.from_numpy(O.grid.mesh_qred(w.mesh)).to(dev)
    nq, n = q.shape[0], 3
    freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
    evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
    vv = torch.zeros((nq, n, 3, 3), dtype=torch.float64, device=dev)
    ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, freq=freq, evec=evec, vv=vv,
                 want_vel=False)
    irr, f2i, _ = phx.irreducible(w.mesh, w.rotations)
    irr_d = torch.from_numpy(irr.astype(np.int32)).to(dev)
    f2i_d = torch.from_numpy(f2i.astype(np.int32)).to(dev)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, w.mesh)
    g_irr = torch.zeros((len(irr), n), dtype=torch.float64, device=dev)
    ctx.gamma(h, freq, evec, irr_d, w.temperature, w.shape, w.sigma_thz, gamma=g_irr)
    g_full = torch.zeros((nq, n), dtype=torch.float64, device=dev)
    ctx.unfold(freq, irr_d, g_irr, f2i_d, out=g_full)
    out = torch.zeros(9, dtype=torch.float64, device=dev)
    for T in (w.temperature, 2.5 * w.temperature):      # second call must not see the first's partials
        ref = ctx.kappa_rta(c.lattice, c.masses, freq, g_full, T, vv=vv)
        phx.kappa_rta_noalloc(c.lattice, c.masses, freq, g_full, T, out, vv=vv)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(3, 3)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        assert np.abs(ref).max() > 0
    ctx.close()
