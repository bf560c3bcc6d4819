"""Learned linewidths on a dense mesh: exact linewidths on a coarse subgrid train an MLP
ensemble (the library's own kernels) that fills the dense mesh; modes where the ensemble
disagrees most, and a held-out part of the subgrid, go to the exact kernel.

Every number is computed by libphx (harmonic, phx_gamma, phx_features, phx_mlp_*, unfold,
conductivity); this module only selects indices and moves arrays between calls.
"""
from __future__ import annotations

import time

import numpy as np


def _timer(torch):
    torch.cuda.synchronize()
    return time.perf_counter()


def subgrid_points(mesh, step):
    """Flat indices of the dense-mesh points whose coordinates are all multiples of step."""
    n1, n2, n3 = mesh
    out = []
    for i in range(n1):
        for j in range(n2):
            for k in range(n3):
                if i % step == 0 and j % step == 0 and k % step == 0:
                    out.append((i * n2 + j) * n3 + k)
    return np.array(out, dtype=np.int64)


def run(ctx, phx, lattice, masses, ifc2_idx, ifc2_val, ifc3_idx, ifc3_val, mesh, step, rotations, temperature,
        shape="gauss", sigma=0.1, f_min=0.01, precision="bf16x3", epochs=3000, lr=3e-3, heldout_frac=0.05,
        uncertainty_pct=95.0, ensemble=4, width=128, depth=3, seed=0, exact_reference=True, residual=True,
        early_stop=True, val_frac=0.1, check_every=50, patience=4, ood_fallback=True):
    """Surrogate linewidths and RTA conductivity on `mesh` trained on the subgrid of spacing
    `step`.  Returns a dict with the conductivities (surrogate, exact when asked, nearest-
    subgrid baseline), errors, timings and counts.

    residual: the network learns log(gamma / WP2) (the phase-space-averaged coupling, smooth in
    the descriptors) instead of log(gamma); gamma = WP2 * exp(prediction).

    early_stop: a seeded val_frac of the training rows is kept out of the gradient and training
    stops once its loss has not improved for `patience` checks of `check_every` epochs (at most
    `epochs`); otherwise exactly `epochs` full-batch Adam steps.

    ood_fallback: q-points with a mode whose descriptors lie outside the range of the training
    rows go to the exact kernel as well (on top of the uncertainty_pct rule)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    n = 3 * len(masses)
    nq = int(np.prod(mesh))
    qh = np.array([((i // (mesh[1] * mesh[2])) / mesh[0], ((i // mesh[2]) % mesh[1]) / mesh[1],
                    (i % mesh[2]) / mesh[2]) for i in range(nq)])
    q = torch.from_numpy(qh).to(dev)
    freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
    evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
    vel = torch.zeros((nq, n, 3), dtype=torch.float64, device=dev)
    vv = torch.zeros((nq, n, 3, 3), dtype=torch.float64, device=dev)
    t = {}
    t0 = _timer(torch)
    ctx.harmonic(lattice, masses, ifc2_idx, np.asarray(ifc2_val).reshape(-1, 9), q, freq=freq, evec=evec, vel=vel,
                 vv=vv)
    irr, f2i, _ = phx.irreducible(mesh, rotations)
    h = ctx.fc3(lattice, masses, ifc3_idx, ifc3_val, mesh)
    t["harmonic"] = _timer(torch) - t0

    sub = set(subgrid_points(mesh, step).tolist())
    train_q = np.array([i for i in irr if int(i) in sub], dtype=np.int32)
    pos = {int(v): k for k, v in enumerate(irr)}
    gamma_irr = torch.zeros((len(irr), n), dtype=torch.float64, device=dev)
    exact_rows = np.zeros(len(irr), dtype=bool)

    # exact linewidths on the subgrid
    t0 = _timer(torch)
    g_train = ctx.gamma(h, freq, evec, torch.from_numpy(train_q).to(dev), temperature, shape, sigma, 2.0, f_min,
                        precision=precision, gamma=torch.zeros((len(train_q), n), dtype=torch.float64, device=dev))
    t["exact_subgrid"] = _timer(torch) - t0
    rows_train = torch.tensor([pos[int(v)] for v in train_q], device=dev)
    gamma_irr[rows_train] = g_train
    exact_rows[rows_train.cpu().numpy()] = True
    train_mask0 = exact_rows.copy()

    # descriptors of every irreducible dense mode
    t0 = _timer(torch)
    irr_d = torch.from_numpy(irr.astype(np.int32)).to(dev)
    feats = ctx.features(mesh, freq, vel, irr_d, temperature, shape, sigma, 2.0, f_min)
    t["features"] = _timer(torch) - t0
    X_all = feats.reshape(-1, 4).contiguous()
    f_all = freq[irr_d.long()].reshape(-1)
    live = (f_all >= f_min).cpu().numpy()

    # training rows: live subgrid modes; a seeded held-out part is kept aside
    tr_rows = np.concatenate([np.arange(r * n, (r + 1) * n) for r in rows_train.cpu().numpy()])
    tr_rows = tr_rows[live[tr_rows]]
    rng = np.random.default_rng(seed)
    n_hold = max(1, int(round(heldout_frac * len(tr_rows))))
    perm = rng.permutation(len(tr_rows))
    hold_rows, fit_rows = tr_rows[perm[:n_hold]], tr_rows[perm[n_hold:]]
    n_val = max(1, int(round(val_frac * len(fit_rows)))) if early_stop else 0   # the last n_val fit rows
    y_all = gamma_irr.reshape(-1)
    wp2_all = X_all[:, 2].contiguous()
    Xf = X_all[torch.from_numpy(fit_rows).to(dev)].contiguous()
    yf = y_all[torch.from_numpy(fit_rows).to(dev)]
    if residual:
        yf = yf / torch.clamp(wp2_all[torch.from_numpy(fit_rows).to(dev)], min=1e-300)
    yf = yf.contiguous()

    def fit(model):
        if early_stop:
            return model.train_es(Xf, yf, n_val, epochs, lr, check_every, patience)
        return model.train(Xf, yf, epochs, lr), epochs

    t0 = _timer(torch)
    model = ctx.mlp(4, width, depth, ensemble, seed)
    final_loss, epochs_run = fit(model)
    # a member whose final loss stays far above the others' has not converged (it would bias the
    # ensemble mean and inflate its spread): train the ensemble again from another seed, twice
    # at most
    for retry in range(2):
        fl = np.asarray(final_loss, dtype=np.float64)
        if ensemble < 2 or fl.max() <= 4.0 * np.median(fl):
            break
        model.close()
        model = ctx.mlp(4, width, depth, ensemble, seed + 1 + retry)
        final_loss, ep = fit(model)
        epochs_run += ep
    t["train"] = _timer(torch) - t0

    t0 = _timer(torch)
    mean, std = model.predict(X_all)
    # rows whose descriptors lie outside the range of the training rows: the network would
    # extrapolate there (typically the acoustic modes closer to Gamma than any subgrid point)
    outside = model.outside(X_all) if ood_fallback else None
    # linewidths (exp of the prediction, times WP2 for the residual target, 0 below f_min) and
    # the per-q-point ensemble spread (infinite where a mode is outside), on the device
    pred_d, score_d = ctx.mlp_reconstruct(n, mean, std, wp2_all if residual else None, f_all.contiguous(), f_min,
                                          outside=outside)
    t["infer"] = _timer(torch) - t0
    score = score_d.cpu().numpy()
    # held-out check (reported, not used by the path)
    hold_d = torch.from_numpy(hold_rows).to(dev)
    hold_err = (torch.abs(pred_d[hold_d] - y_all[hold_d]) / y_all[hold_d]).cpu().numpy()

    # exact fallback on the q-points outside the network's domain, and on those whose most
    # uncertain mode ranks in the top (100 - uncertainty_pct) % of the other q-points outside
    # the subgrid
    cand = np.array([k for k in range(len(irr)) if not train_mask0[k]], dtype=np.int64)
    ood, pick = fallback_rows(score, cand, uncertainty_pct)
    fb_q = sorted(int(irr[k]) for k in np.concatenate([ood, pick]))
    t0 = _timer(torch)
    if fb_q:
        fb = np.array(fb_q, dtype=np.int32)
        g_fb = ctx.gamma(h, freq, evec, torch.from_numpy(fb).to(dev), temperature, shape, sigma, 2.0, f_min,
                         precision=precision, gamma=torch.zeros((len(fb), n), dtype=torch.float64, device=dev))
        rows_fb = torch.tensor([pos[v] for v in fb_q], device=dev)
        gamma_irr[rows_fb] = g_fb
        exact_rows[rows_fb.cpu().numpy()] = True
    t["fallback"] = _timer(torch) - t0

    g_sur = gamma_irr.clone()
    pred_t = pred_d.reshape(len(irr), n)
    mask = torch.from_numpy(~exact_rows).to(dev)
    g_sur[mask] = pred_t[mask]
    f2i_d = torch.from_numpy(f2i.astype(np.int32)).to(dev)

    def kappa_of(g_irr):
        gf = ctx.unfold(freq, irr_d, g_irr.contiguous(), f2i_d, out=torch.zeros((nq, n), dtype=torch.float64,
                                                                             device=dev))
        return ctx.kappa_rta(lattice, masses, freq, gf, temperature, vv=vv, f_min=f_min)

    k_sur = kappa_of(g_sur)

    # the method without the network at the same cost: nearest subgrid point, same band
    coords = np.array([((v // (mesh[1] * mesh[2])), (v // mesh[2]) % mesh[1], v % mesh[2]) for v in irr])
    near = (np.rint(coords / step).astype(int) * step) % np.array(mesh)
    near_idx = (near[:, 0] * mesh[1] + near[:, 1]) * mesh[2] + near[:, 2]
    g_train_full = ctx.unfold(freq, torch.from_numpy(train_q).to(dev), g_train.contiguous(),
                              torch.from_numpy(_orbit_map(mesh, rotations, train_q, phx)).to(dev),
                              out=torch.zeros((nq, n), dtype=torch.float64, device=dev))
    g_base = g_train_full[torch.from_numpy(near_idx).to(dev)]
    train_mask = np.zeros(len(irr), dtype=bool)
    train_mask[rows_train.cpu().numpy()] = True
    g_base[torch.from_numpy(train_mask).to(dev)] = g_train
    k_base = kappa_of(g_base)

    # the method without the network: the exact path on the coarse subgrid mesh itself
    t0 = _timer(torch)
    cmesh = tuple(int(m // step) for m in mesh)
    k_coarse = _coarse_kappa(ctx, phx, lattice, masses, ifc2_idx, ifc2_val, ifc3_idx, ifc3_val, cmesh, rotations,
                             temperature, shape, sigma, f_min, precision)
    t["coarse_mesh_exact"] = _timer(torch) - t0

    out = dict(kappa_surrogate=k_sur, kappa_interp=k_base, kappa_coarse=k_coarse, timings=t, final_loss=final_loss,
               heldout_median_rel_err=float(np.median(hold_err)), heldout_max_rel_err=float(hold_err.max()),
               n_irr=len(irr), n_train_q=len(train_q), n_fallback_q=len(fb_q), n_outside_q=len(ood),
               n_train_rows=len(fit_rows) - n_val,
               n_val_rows=n_val, n_heldout_rows=len(hold_rows), epochs_run=epochs_run)
    if exact_reference:
        t0 = _timer(torch)
        g_ex = ctx.gamma(h, freq, evec, irr_d, temperature, shape, sigma, 2.0, f_min, precision=precision,
                         gamma=torch.zeros((len(irr), n), dtype=torch.float64, device=dev))
        t["exact_full"] = _timer(torch) - t0
        k_ex = kappa_of(g_ex)
        out["kappa_exact"] = k_ex
        nrm = np.linalg.norm(k_ex)
        out["kappa_rel_err_surrogate"] = float(np.linalg.norm(k_sur - k_ex) / nrm)
        out["kappa_rel_err_interp"] = float(np.linalg.norm(k_base - k_ex) / nrm)
        out["kappa_rel_err_coarse"] = float(np.linalg.norm(k_coarse - k_ex) / nrm)
        fr = freq.cpu().numpy()[irr]
        out["triplets_exact"] = int((fr >= f_min).sum()) * nq * n * n
    model.close()
    return out


def fallback_rows(score, cand, uncertainty_pct):
    """Rows (irreducible q-points) sent back to the exact kernel among the candidates `cand`:
    every one whose score is infinite (a mode outside the network's domain), and the
    (100 - uncertainty_pct) % of all candidates with the largest finite scores (ensemble
    spread; ties keep candidate order).  Returns (outside, by_spread)."""
    cand = np.asarray(cand, dtype=np.int64)
    score = np.asarray(score, dtype=np.float64)
    ood = cand[np.isinf(score[cand])]
    rest = cand[~np.isinf(score[cand])]
    n_fb = int(np.ceil((100.0 - uncertainty_pct) / 100.0 * len(cand)))
    pick = rest[np.argsort(-score[rest], kind="stable")[:n_fb]] if n_fb > 0 else rest[:0]
    return ood, pick


def _orbit_map(mesh, rotations, reps, phx):
    """full_to_irr for the subgrid representatives: each mesh point mapped to the position in
    `reps` of its orbit's representative (points outside the subgrid map to 0; unused)."""
    irr, f2i, _ = phx.irreducible(mesh, rotations)
    pos = {int(v): k for k, v in enumerate(reps)}
    return np.array([pos.get(int(irr[f2i[i]]), 0) for i in range(len(f2i))], dtype=np.int32)


def _coarse_kappa(ctx, phx, lattice, masses, ifc2_idx, ifc2_val, ifc3_idx, ifc3_val, mesh, rotations, temperature,
                  shape, sigma, f_min, precision):
    """RTA conductivity computed exactly on `mesh` (harmonic, linewidths, unfold, kappa)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    n = 3 * len(masses)
    nq = int(np.prod(mesh))
    qh = np.array([((i // (mesh[1] * mesh[2])) / mesh[0], ((i // mesh[2]) % mesh[1]) / mesh[1],
                    (i % mesh[2]) / mesh[2]) for i in range(nq)])
    freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
    evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
    vv = torch.zeros((nq, n, 3, 3), dtype=torch.float64, device=dev)
    ctx.harmonic(lattice, masses, ifc2_idx, np.asarray(ifc2_val).reshape(-1, 9), torch.from_numpy(qh).to(dev),
                 freq=freq, evec=evec, vv=vv, want_vel=False)
    irr, f2i, _ = phx.irreducible(mesh, rotations)
    h = ctx.fc3(lattice, masses, ifc3_idx, ifc3_val, mesh)
    irr_d = torch.from_numpy(irr.astype(np.int32)).to(dev)
    g = ctx.gamma(h, freq, evec, irr_d, temperature, shape, sigma, 2.0, f_min, precision=precision,
                  gamma=torch.zeros((len(irr), n), dtype=torch.float64, device=dev))
    gf = ctx.unfold(freq, irr_d, g, torch.from_numpy(f2i.astype(np.int32)).to(dev),
                    out=torch.zeros((nq, n), dtype=torch.float64, device=dev))
    k = ctx.kappa_rta(lattice, masses, freq, gf, temperature, vv=vv, f_min=f_min)
    h.close()
    return k
