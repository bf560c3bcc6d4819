"""Batched jobs (many crystals in one captured graph) against the single-job path and the
oracle: same linewidths and conductivities, identical results on graph replay."""
import numpy as np
import pytest

import oracle as O
import phx_inputs as P

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

SIZES = [(1, 4), (2, 3), (3, 4), (4, 3), (6, 2), (8, 3), (12, 2), (16, 2)]    # (atoms, mesh edge)


@pytest.fixture(scope="module")
def phx():
    import paper_2602_23728_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(phx):
    c = phx.Context(0)
    yield c
    c.close()


def _job(ctx, phx, na, m, seed, T):
    import torch
    dev = torch.device("cuda:0")
    c = P.random_masses(P.fcc_primitive_multiple(5.26, P.most_cubic_factorisation(na)), 39.95, 83.8, seed=seed)
    pot = P.LennardJones()
    mesh = (m, m, m)
    f2, f3 = P.ifc2_lj(c, pot), P.ifc3_lj(c, pot)
    n = 3 * na
    nq = m ** 3
    q = torch.from_numpy(O.grid.mesh_qred(mesh)).to(dev)
    freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
    evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
    vv = torch.zeros((nq, n, 3, 3), dtype=torch.float64, device=dev)
    ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, freq=freq, evec=evec, vv=vv,
                 want_vel=False)
    irr, f2i, _ = phx.irreducible(mesh, P.identity_rotation())
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    return dict(fc3=h, freq=freq, evec=evec, irr=irr, irr_dev=torch.from_numpy(irr.astype(np.int32)).to(dev),
                T=T, shape="gauss", sigma=0.1, window=2.0, f_min=0.01,
                gamma=torch.zeros((len(irr), n), dtype=torch.float64, device=dev),
                vv=vv, full_to_irr=torch.from_numpy(f2i.astype(np.int32)).to(dev),
                gamma_full=torch.zeros((nq, n), dtype=torch.float64, device=dev),
                kappa=torch.zeros(9, dtype=torch.float64, device=dev), volume=c.volume,
                crystal=c, f3=f3, mesh=mesh)


@pytest.fixture(scope="module")
def jobs(ctx, phx):
    rng = np.random.default_rng(3)
    return [_job(ctx, phx, na, m, 100 + k, float(rng.uniform(20, 80))) for k, (na, m) in enumerate(SIZES)]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_batched_matches_single_jobs_and_replays(ctx, phx, jobs, prec):
    import torch
    import torch.cuda
    tuned = ctx.gamma_batched(jobs, precision=prec)
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for q, ch, sd in tuned:           # the autotuner's choices per job, written back
        assert 8 <= q <= 128 and ch in (0, 1) and 0 <= sd <= sms // 2
    first = [j["gamma"].cpu().numpy().copy() for j in jobs]
    kap = [j["kappa"].cpu().numpy().copy() for j in jobs]
    for j in jobs:
        j["gamma"].zero_()
        j["kappa"].zero_()
    # replay of the cached graph, with the tuned choices passed back in (same launches)
    again = ctx.gamma_batched(jobs, precision=prec, q_tiles=[t[0] for t in tuned], chain=[t[1] for t in tuned],
                              side_sms=[t[2] for t in tuned])
    assert again == tuned
    torch.cuda.synchronize()
    for k, j in enumerate(jobs):
        assert np.array_equal(j["gamma"].cpu().numpy(), first[k]) or \
            np.abs(j["gamma"].cpu().numpy() - first[k]).max() <= 1e-12 * np.abs(first[k]).max()
        single = ctx.gamma(j["fc3"], j["freq"], j["evec"], j["irr_dev"], j["T"], precision=prec,
                           gamma=torch.zeros_like(j["gamma"]))
        torch.cuda.synchronize()
        s = single.cpu().numpy()
        assert np.abs(first[k] - s).max() <= 1e-6 * max(np.abs(s).max(), 1e-30)
        # conductivity inside the graph = unfold + kappa on the same linewidths
        gf = ctx.unfold(j["freq"], j["irr_dev"], j["gamma"], j["full_to_irr"],
                        out=torch.zeros_like(j["gamma_full"]))
        K = ctx.kappa_rta(j["crystal"].lattice, j["crystal"].masses, j["freq"], gf, j["T"], vv=j["vv"])
        assert np.linalg.norm(kap[k].reshape(3, 3) - K) <= 1e-10 * max(np.linalg.norm(K), 1e-30)


def test_batched_small_jobs_match_oracle(ctx, phx, jobs):
    import torch
    ctx.gamma_batched(jobs, precision="bf16x3", q_tiles=[8] * len(jobs))
    torch.cuda.synchronize()
    for j in jobs[:3]:
        c = j["crystal"]
        fc3 = O.anharmonic.FC3(j["f3"].idx, j["f3"].val, c.masses)
        freq = j["freq"].cpu().numpy()
        evec = j["evec"].cpu().numpy()
        go = O.anharmonic.gamma(fc3, j["mesh"], freq, evec, j["irr"], j["T"], "gauss", 0.1)
        g = j["gamma"].cpu().numpy()
        big = go > 1e-3 * go.max()
        assert go.max() > 0
        assert (np.abs(g - go)[big] / go[big]).max() < 1e-4


def test_batched_side_stream_share_changes_no_result(ctx, phx, jobs):
    """The side-stream share (a tuned parameter) moves the fold and Fourier GEMM to other SMs
    and changes no arithmetic: one stream and 24 side SMs agree to the FP64 accumulation order."""
    import torch
    out = []
    for sd in (0, 24):
        ctx.gamma_batched(jobs, precision="bf16x3", q_tiles=[16] * len(jobs), chain=[-1] * len(jobs),
                          side_sms=[sd] * len(jobs))
        torch.cuda.synchronize()
        out.append([j["gamma"].cpu().numpy().copy() for j in jobs])
    for a, b in zip(*out):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-30)
