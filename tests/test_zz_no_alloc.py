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


def test_kappa_noalloc_many_blocks_then_fewer():
    """More than 2048 modes (several partial rows summed in a fixed order), per-mode velocities,
    against the oracle's Eq. (rta); then a smaller call that uses fewer rows than the last one;
    then the velocity-product path on the large case."""
    import torch
    import paper_2602_23728_gb300 as phx
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(21)
    c = P.fcc_monatomic_5().crystal
    out = torch.zeros(9, dtype=torch.float64, device=dev)
    for nq, n in ((300, 24), (7, 6)):
        f = rng.uniform(0.0, 3.0, size=(nq, n))
        f[0, :2] = 0.001                                   # below f_min: skipped
        g = rng.uniform(0.05, 0.5, size=(nq, n))
        v = rng.normal(size=(nq, n, 3))
        ref = O.transport.kappa_rta(f, v, g, 40.0, c.volume, f_min=0.01)
        phx.kappa_rta_noalloc(c.lattice, c.masses, torch.from_numpy(f).to(dev), torch.from_numpy(g).to(dev), 40.0,
                              out, vel=torch.from_numpy(v).to(dev))
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(3, 3)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        if nq == 300:
            vv = np.einsum("qna,qnb->qnab", v, v)
            phx.kappa_rta_noalloc(c.lattice, c.masses, torch.from_numpy(f).to(dev), torch.from_numpy(g).to(dev),
                                  40.0, out, vv=torch.from_numpy(vv).to(dev))
            torch.cuda.synchronize()
            assert np.linalg.norm(out.cpu().numpy().reshape(3, 3) - ref) <= 1e-12 * np.linalg.norm(ref)
    with pytest.raises(ValueError):
        phx.kappa_rta_noalloc(c.lattice, c.masses, torch.zeros((2, 3), device=dev, dtype=torch.float64),
                              torch.zeros((2, 3), device=dev, dtype=torch.float64), 40.0,
                              torch.zeros(4, device=dev, dtype=torch.float64),
                              vel=torch.zeros((2, 3, 3), device=dev, dtype=torch.float64))
