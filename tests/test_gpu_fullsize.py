"""Full-size parity at the bench workload (32-atom mass-disordered LJ fcc, 96 modes, 8x8x8
mesh, 260 irreducible q, 50 K, Gaussian 0.1 THz), in the launch configuration bench.py times:
the library's own harmonic phonons, BF16x3 linewidths of every irreducible mode (chained
tensor-core kernel), unfolding and Eq. (rta), against the FP64 oracle's linewidths and
conductivity stored under tests/golden/ (written by tests/golden/make_golden_kappa.py from
oracle/ only).  Bars: gamma within 1e-4 on modes above 1e-3 of the maximum, kappa within
1e-5 (Frobenius-relative)."""
import os

import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu]
HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden():
    from test_golden_files import read_kappa_file
    return read_kappa_file(os.path.join(HERE, "fcc32_mesh8_kappa.txt"))


@pytest.mark.parametrize("prec,g_bar,k_bar", [("bf16x3", 1e-4, 1e-5), ("tf32", 2e-2, 1e-3)])
def test_fcc32_all_modes_and_kappa_vs_oracle(prec, g_bar, k_bar):
    import torch
    import paper_2602_23728_gb300 as phx
    digest, k_ref, rows = _golden()
    w = P.fcc_massdisorder_32()
    f2, f3 = w.ifc2(), w.ifc3()
    assert digest == P.workload_digest(w, f2, f3)
    c = w.crystal
    dev = torch.device("cuda:0")
    ctx = phx.Context(0)
    try:
        q = torch.from_numpy(O.grid.mesh_qred(w.mesh)).to(dev)
        nq, n = q.shape[0], 96
        freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
        evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
        vv = torch.zeros((nq, n, 3, 3), dtype=torch.float64, device=dev)
        ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, freq=freq, evec=evec, vv=vv,
                     want_vel=False)
        irr, f2i, _ = phx.irreducible(w.mesh, w.rotations)
        h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, w.mesh)
        irr_d = torch.from_numpy(irr.astype(np.int32)).to(dev)
        g = torch.zeros((len(irr), n), dtype=torch.float64, device=dev)
        ctx.gamma(h, freq, evec, irr_d, w.temperature, w.shape, w.sigma_thz, w.window, w.f_min_thz, precision=prec,
                  gamma=g)
        gf = ctx.unfold(freq, irr_d, g, torch.from_numpy(f2i.astype(np.int32)).to(dev),
                        out=torch.zeros((nq, n), dtype=torch.float64, device=dev))
        K = ctx.kappa_rta(c.lattice, c.masses, freq, gf, w.temperature, vv=vv, f_min=w.f_min_thz)
        fr = freq.cpu().numpy()
        gh = np.array([O.anharmonic.degenerate_average(fr[i], g[s].cpu().numpy()) for s, i in enumerate(irr)])
        ref = rows[:, 2].reshape(len(irr), n)
        assert np.array_equal(rows[::n, 0].astype(int), irr)
        big = ref > 1e-3 * ref.max()
        g_err = float((np.abs(gh - ref)[big] / ref[big]).max())
        k_err = float(np.linalg.norm(K - k_ref) / np.linalg.norm(k_ref))
        print(f"{prec}: all {big.sum()} modes gamma max rel err {g_err:.2e}, kappa rel err {k_err:.2e}")
        assert g_err < g_bar
        assert k_err < k_bar
    finally:
        ctx.close()
