"""Isotope scattering on the GPU (phx_gamma_isotope) against the oracle of Eq. (isotope) with
shared eigenvectors: two-atom cell on a ragged mesh, both broadenings, device buffers, and the
Gamma point of a disordered supercell."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def ctx():
    import paper_2602_23728_gb300 as m
    c = m.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape", ["gauss", "lorentz"])
def test_isotope_matches_oracle(ctx, shape):
    c = P.fcc_primitive_multiple(5.26, (2, 1, 1))
    c = P.Crystal(c.lattice, c.positions, np.array([39.95, 83.8]), "fcc2")
    f2 = P.ifc2_lj(c, P.LennardJones())
    mesh = (3, 4, 5)
    q = O.grid.mesh_qred(mesh)
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, want_vel=False,
                                    want_vv=False)
    irr = np.arange(0, q.shape[0], 7, dtype=np.int32)
    g = np.array([0.12, 0.03])
    got = ctx.gamma_isotope(freq, evec, irr, g, shape=shape, sigma=0.2)
    ref = O.isotope.gamma_iso(freq, evec, irr, g, shape, 0.2)
    assert ref.max() > 0
    assert np.abs(got - ref).max() <= 1e-11 * ref.max()


def test_isotope_device_buffers_and_gamma_cell(ctx):
    import torch
    c = P.random_masses(P.fcc_primitive_multiple(5.26, (5, 4, 4)), 39.95, 83.8, seed=2)
    f2, _ = P.ifc_lj_vectorised(c, P.LennardJones())
    freq, evec, _, _ = ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), np.zeros((1, 3)),
                                    want_vel=False, want_vv=False)
    g = np.full(c.n_atoms, O.isotope.g_factor([0.5, 0.5], [39.95, 83.8]))
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(freq).to(dev)
    ed = torch.from_numpy(evec).to(dev)
    irr = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.zeros((1, freq.shape[1]), dtype=torch.float64, device=dev)
    ctx.gamma_isotope(fd, ed, irr, g, shape="lorentz", sigma=0.1, gamma=out)
    torch.cuda.synchronize()
    ref = O.isotope.gamma_iso(freq, evec, [0], g, "lorentz", 0.1)
    assert ref.max() > 0
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-11 * ref.max()
