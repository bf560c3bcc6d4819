#!/usr/bin/env python
"""Throughput of the three-phonon scattering hot path on GB300, in phonon triplets/s.

One step = the whole path on the 32-atom mass-disordered LJ fcc cell (96 modes), 8x8x8
mesh, 50 K, Gaussian 0.1 THz: harmonic phonons on every mesh point (FP64 eigensolver),
linewidths of every mode of the 260 irreducible q-points (tensor-core contraction),
unfolding, RTA conductivity.  A triplet is one (lambda, q', nu', nu'') element with
lambda an irreducible mode above f_min (both scattering processes come from it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|tf32|fp64]
    python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample

Prints one JSON line (rank 0).  Under torchrun every rank runs its own replica of the
workload on its own GPU (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phonon triplets/s (V3+gamma) on 1 GB300, mixed/batched vs FP64 path, at stated kappa error"
UNIT = "triplets/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
# kernel classes that run on the tensor cores (their recorded flops are algorithmic: 8 flops per
# useful complex multiply-add, padding excluded)
TENSOR_CLASSES = ("dft", "chain", "gemm_e2", "gemm_e1_gamma", "cell_gemm")
# DRAM bytes per launch measured by ncu, with the hash of the CUDA sources they were taken on
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
KERNEL_SOURCES = ("chain_tc.cuh", "common.h", "gamma_common.cuh", "gamma_tc.cu", "tc_ptx.cuh")
GOLDEN_KAPPA = os.path.join(ROOT, "tests", "golden", "fcc32_mesh8_kappa.txt")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2602_23728_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, precision, workload):
    """ncu DRAM bytes per launch of a kernel class on a workload, or None when no capture was
    taken on the current kernel sources."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    src = kernel_source_hash()
    with open(TRAFFIC_FILE) as fh:
        for line in fh:
            f = line.split()
            if len(f) == 5 and not line.startswith("#") and f[:3] == [workload, kernel, precision] and f[4] == src:
                return float(f[3])
    return None


def tensor_peak(peaks, precision, sustained=True):
    """Dense tensor peak in TFLOP/s of FP32-equivalent products for a precision (None for FP64)."""
    bf16 = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops", peaks.get("bf16_tflops"))
    if precision == "bf16x3":
        return bf16 / 3.0, "bf16 %s / 3 (three bf16 products per FP32-equivalent product)" % (
            "sustained" if sustained else "burst")
    if precision == "tf32":
        return bf16 * NOMINAL_TF32_OVER_BF16, "bf16 %s x nominal tf32/bf16 (1.1/2.25)" % (
            "sustained" if sustained else "burst")
    return None, "FP64 CUDA-core path"


def new_context(phx, device, args):
    """Library context with the run's options."""
    ctx = phx.Context(device)
    ctx.set_option("pair", args.pair)
    ctx.set_option("vel_fp32", args.vel_fp32)
    return ctx


def pair_count(iq, mesh, pair=True):
    """q' contracted for irreducible q: every mesh point, or with exchange pairs one per
    unordered {q', q''} ((nq + n_self) / 2, n_self = the q' with 2 q' = -q mod G)."""
    nq = int(np.prod(mesh))
    if not pair:
        return nq
    k = (iq // (mesh[1] * mesh[2]), (iq // mesh[2]) % mesh[1], iq % mesh[2])
    n_self = 1
    for d in range(3):
        n_self *= 1 if mesh[d] % 2 else (0 if k[d] % 2 else 2)
    return (nq + n_self) // 2


def roofline_of(prof, steps, ms_step, precision, peaks, src, workload, sm_share=None):
    """Roofline of the kernel class with the most device time in a profiled pass of `steps`
    steps: tensor-bound classes against the tensor peak of the precision (algorithmic flops),
    with the HBM figure (algorithmic bytes over the copy bandwidth) as a second field.
    sm_share: {class: (SMs the class runs on, SMs of the GPU)} for classes confined to part of
    the GPU (the chained kernel next to the side stream); their line adds the fraction of the
    peak of those SMs."""
    per = {k: v for k, v in prof.items() if k != "launches" and v[1] > 0}
    if not per:
        return None
    name = max(per, key=lambda k: per[k][0])
    tot_ms, nl, fl, by = per[name]
    t = tot_ms / 1e3
    peak, note = tensor_peak(peaks, precision)
    hbm = {"achieved": by / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": by / t / 1e9 / peaks["hbm_gbs"], "bytes_per_launch": by / nl,
           "peak_source": f"{src}: copy bandwidth"}
    traffic = measured_traffic(name, precision, workload)
    if name in TENSOR_CLASSES and peak:
        ach = fl / t / 1e12
        roof = {"bound": "tensor", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic, "peak_source": f"{src}: {note}", "hbm": hbm}
    else:
        roof = {"bound": "hbm", "kernel": name, "achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s",
                "frac": hbm["frac"], "traffic": traffic, "peak_source": hbm["peak_source"]}
    roof.update({"algorithmic_flops_per_launch": fl / nl, "algorithmic_bytes_per_launch": by / nl,
                 "launches_per_step": nl / steps, "avg_launch_ms": tot_ms / nl,
                 "share_of_step": tot_ms / steps / ms_step})
    if sm_share and name in sm_share and sm_share[name][0] < sm_share[name][1]:
        used, total = sm_share[name]
        roof.update({"sms": used, "sms_total": total, "frac_of_its_sms_peak": roof["frac"] * total / used,
                     "sms_note": f"runs on {used} of {total} SMs while the fold and Fourier GEMM of the next q' "
                                 f"tile run on the other {total - used} (frac is against the whole GPU's peak)"})
    return roof


def golden_kappa(w, f2, f3):
    """The oracle's RTA conductivity stored under tests/golden/ for this workload, or None."""
    import phx_inputs as P
    if not os.path.exists(GOLDEN_KAPPA):
        return None
    digest, kappa = None, None
    with open(GOLDEN_KAPPA) as fh:
        for line in fh:
            if line.startswith("# inputs "):
                digest = line.split()[2]
            elif line.startswith("kappa "):
                kappa = np.array([float(x) for x in line.split()[1:]]).reshape(3, 3)
                break
    if kappa is None or digest != P.workload_digest(w, f2, f3):
        return None
    return kappa


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return PEAKS_FALLBACK, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- workload

class Workload:
    """Inputs of the 32-atom / 8x8x8 workload, resident on the device."""

    def __init__(self, phx, ctx, precision, device, mesh=(8, 8, 8)):
        import torch
        import phx_inputs as P
        self.torch = torch
        self.w = w = P.fcc_massdisorder_32(mesh=tuple(mesh))
        self.f2, self.f3 = w.ifc2(), w.ifc3()
        f3 = self.f3
        self.f2val = self.f2.val.reshape(-1, 9)
        c = w.crystal
        self.c = c
        self.n = 3 * c.n_atoms
        self.precision = precision
        self.ctx = ctx
        self.h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, w.mesh)
        self.irr, self.f2i, _ = phx.irreducible(w.mesh, w.rotations)
        nq = int(np.prod(w.mesh))
        self.nq = nq
        self.q_host = np.array([(i // (w.mesh[1] * w.mesh[2]) / w.mesh[0], (i // w.mesh[2]) % w.mesh[1] / w.mesh[1],
                                 i % w.mesh[2] / w.mesh[2]) for i in range(nq)])
        dev = device
        f64 = torch.float64
        self.q = torch.from_numpy(self.q_host).to(dev)
        self.freq = torch.zeros((nq, self.n), dtype=f64, device=dev)
        self.evec = torch.zeros((nq, self.n, self.n), dtype=torch.complex128, device=dev)
        self.vv = torch.zeros((nq, self.n, 3, 3), dtype=f64, device=dev)
        self.irr_d = torch.from_numpy(self.irr.astype(np.int32)).to(dev)
        self.f2i_d = torch.from_numpy(self.f2i.astype(np.int32)).to(dev)
        self.g_irr = torch.zeros((len(self.irr), self.n), dtype=f64, device=dev)
        self.g_full = torch.zeros((nq, self.n), dtype=f64, device=dev)
        self.kappa = None

    def limit_irreducible(self, k):
        """Small-case mode for profiler captures: only the first k irreducible q-points."""
        self.irr = self.irr[:k]
        self.irr_d = self.irr_d[:k].contiguous()
        self.g_irr = self.g_irr[:k].contiguous()
        self.f2i = np.minimum(self.f2i, k - 1).astype(np.int32)
        self.f2i_d = self.torch.from_numpy(self.f2i).to(self.irr_d.device)

    def step(self, precision=None):
        prec = precision or self.precision
        w, c, ctx = self.w, self.c, self.ctx
        ctx.harmonic(c.lattice, c.masses, self.f2.idx, self.f2val, self.q, freq=self.freq, evec=self.evec,
                     vel=None, vv=self.vv, want_vel=False)
        ctx.gamma(self.h, self.freq, self.evec, self.irr_d, w.temperature, w.shape, w.sigma_thz, w.window,
                  w.f_min_thz, precision=prec, gamma=self.g_irr)
        ctx.unfold(self.freq, self.irr_d, self.g_irr, self.f2i_d, out=self.g_full)
        self.kappa = ctx.kappa_rta(c.lattice, c.masses, self.freq, self.g_full, w.temperature, vv=self.vv,
                                   f_min=w.f_min_thz)
        return self.kappa

    def triplets(self):
        f = self.freq.cpu().numpy()
        valid = (f[self.irr] >= self.w.f_min_thz).sum()
        return int(valid) * self.nq * self.n * self.n

    def triplets_evaluated(self, pair):
        """Triplets the contractions evaluate: with exchange pairs about half of triplets()."""
        f = self.freq.cpu().numpy()
        return sum(int((f[iq] >= self.w.f_min_thz).sum()) * pair_count(int(iq), self.w.mesh, pair)
                   for iq in self.irr) * self.n * self.n

    # ---- end to end through the public API with host (pinned) buffers
    def step_host(self, bufs):
        w, c, ctx = self.w, self.c, self.ctx
        ctx.harmonic(c.lattice, c.masses, self.f2.idx, self.f2val, bufs["q"], freq=bufs["freq"], evec=bufs["evec"],
                     vel=None, vv=bufs["vv"], want_vel=False)
        ctx.gamma(self.h, bufs["freq"], bufs["evec"], bufs["irr"], w.temperature, w.shape, w.sigma_thz, w.window,
                  w.f_min_thz, precision=self.precision, gamma=bufs["g_irr"])
        ctx.unfold(bufs["freq"], bufs["irr"], bufs["g_irr"], bufs["f2i"], out=bufs["g_full"])
        return ctx.kappa_rta(c.lattice, c.masses, bufs["freq"], bufs["g_full"], w.temperature, vv=bufs["vv"],
                             f_min=w.f_min_thz)

    def host_buffers(self):
        torch = self.torch

        keep = []

        def pinned(shape, dtype):
            t = torch.zeros(shape, dtype=dtype).pin_memory()
            keep.append(t)               # the numpy view does not own the pinned memory
            return t.numpy()
        n, nq = self.n, self.nq
        b = {"q": pinned((nq, 3), torch.float64), "freq": pinned((nq, n), torch.float64),
             "evec": pinned((nq, n, n), torch.complex128), "vv": pinned((nq, n, 3, 3), torch.float64),
             "irr": pinned((len(self.irr),), torch.int32), "f2i": pinned((nq,), torch.int32),
             "g_irr": pinned((len(self.irr), n), torch.float64), "g_full": pinned((nq, n), torch.float64)}
        b["_keep"] = keep
        b["q"][:] = self.q_host
        b["irr"][:] = self.irr
        b["f2i"][:] = self.f2i
        return b

    def host_bytes(self, b):
        """H2D and D2H bytes one host-buffer step moves (counted from the arrays copied)."""
        ifc2 = self.f2.idx.nbytes + self.f2val.nbytes
        h2d = (b["q"].nbytes + ifc2 + b["freq"].nbytes + b["evec"].nbytes + b["irr"].nbytes       # harmonic, gamma
               + b["freq"].nbytes + b["irr"].nbytes + b["g_irr"].nbytes + b["f2i"].nbytes        # unfold
               + b["freq"].nbytes + b["vv"].nbytes + b["g_full"].nbytes)                          # kappa
        d2h = (b["freq"].nbytes + b["evec"].nbytes + b["vv"].nbytes + 4                           # harmonic (+status)
               + b["g_irr"].nbytes + 4 + b["g_full"].nbytes + 72)
        return int(h2d), int(d2h)


# ----------------------------------------------------------------------------- oracle timing

def oracle_sample(n_qp=None, seed_q=1):
    """FP64 oracle linewidths of one irreducible q-point (all or n_qp of the q'); returns
    (seconds, triplets, description).  The harmonic part is prepared outside the clock."""
    import oracle as O
    import phx_inputs as P
    w = P.fcc_massdisorder_32()
    f2, f3 = w.ifc2(), w.ifc3()
    c = w.crystal
    q = O.grid.mesh_qred(w.mesh)
    freq, evec, _ = O.harmonic.solve(f2.idx, f2.val, c.masses, c.lattice, q)
    fc3 = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
    irr, _, _ = O.grid.irreducible(w.mesh, w.rotations)
    iq = int(irr[seed_q])
    mesh = w.mesh
    nq = q.shape[0]
    if n_qp is None or n_qp >= nq:
        t0 = time.perf_counter()
        O.anharmonic.gamma(fc3, mesh, freq, evec, [iq], w.temperature, w.shape, w.sigma_thz)
        dt = time.perf_counter() - t0
        n_q1 = nq
    else:
        # the oracle's per-pair steps for a bounded set of q' (same arithmetic as its gamma)
        kint = O.grid.mesh_int(mesh)
        nocc = O.occupation.bose(freq, w.temperature)
        t0 = time.perf_counter()
        acc = np.zeros(freq.shape[1])
        for iqp in range(n_qp):
            iqpp = int(O.grid.mesh_index(-(kint[iq] + kint[iqp]), mesh))
            V = O.anharmonic.v3(fc3, evec[iq], q[iqp], evec[iqp], -(q[iq] + q[iqp]), evec[iqpp])
            W = O.anharmonic.pair_weights(freq[iq], freq[iqp], freq[iqpp], nocc[iqp], nocc[iqpp], w.shape,
                                          w.sigma_thz, w.f_min_thz, w.window)
            acc += np.einsum("ijk,ijk->i", np.abs(V) ** 2, W)
        dt = time.perf_counter() - t0
        n_q1 = n_qp
    n = freq.shape[1]
    valid = int((freq[iq] >= w.f_min_thz).sum())
    trip = valid * n_q1 * n * n
    desc = f"oracle gamma of irreducible q-point {iq} over {n_q1} of {nq} q' (1/{len(irr)} of the irreducible set)"
    return dt, trip, desc


def reduce_over_ranks(ms, units, world, dist=None, device="cpu"):
    """Whole-job timing of independent replicas: (max step time over ranks in ms, total units
    over ranks).  The reported value is units / (ms / 1e3).  With world == 1 no collective is
    made; otherwise the process group of `dist` reduces a small tensor on `device` (NCCL on
    the GPU, gloo on the host)."""
    if world <= 1:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count()


# ----------------------------------------------------------------------------- arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_qp = args.ref_qp
    dts, trip = [], 0
    for i in range(args.warmup + args.steps):
        dt, trip, desc = oracle_sample(n_qp=n_qp)
        if i >= args.warmup:
            dts.append(dt)
    ms = 1e3 * float(np.mean(dts))
    val = trip / (ms / 1e3)
    cores = blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fcc32-massdis-mesh8 (32-atom LJ fcc, 96 modes, 8x8x8, 50 K, Gauss 0.1 THz)",
                       "sample": desc},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_phx(args):
    import torch
    import torch.distributed as dist
    import paper_2602_23728_gb300 as phx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    ctx = new_context(phx, local, args)
    wl = Workload(phx, ctx, args.precision, device)
    if args.irr_limit > 0:
        wl.limit_irreducible(args.irr_limit)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        wl.step()
    barrier()
    trip = wl.triplets()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile_enable(False)            # no per-launch events in the timed loop; zeroes the launch count
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            wl.step()
        ev1.record(stream)
        barrier()
    launches = ctx.profile_read()["launches"]
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max, trip_all = reduce_over_ranks(ms, trip, world, dist, device)
    value = trip_all / (ms_max / 1e3)
    kappa = wl.kappa.copy()
    # per-kernel-class times from one separate step with events around every launch
    ctx.profile_enable(True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    wl.step()
    pe1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms_prof = pe0.elapsed_time(pe1)

    # end to end: the same step through the API with pinned host buffers
    bufs = wl.host_buffers()
    wl.step_host(bufs)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        wl.step_host(bufs)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms, _ = reduce_over_ranks(e2e_ms, trip, world, dist, device)
    h2d, d2h = wl.host_bytes(bufs)

    # roofline of the kernel class with the most device time (events of the profiled step)
    peaks, src = load_peaks()
    sms_total = torch.cuda.get_device_properties(device).multi_processor_count
    side = ctx.get_option("side_sms")
    roof = roofline_of(prof, 1, ms_prof, args.precision, peaks, src, "fcc32",
                       sm_share={"chain": (sms_total - side, sms_total)})
    # the whole step's contraction: 16 n flops per evaluated triplet (two complex contractions of
    # n terms, 8 flops per complex multiply-add) over the step time, against the same tensor peak
    peak_t, _ = tensor_peak(peaks, args.precision)
    trip_eval = wl.triplets_evaluated(bool(args.pair))
    step_fl = 16.0 * wl.n * trip_eval
    step_contraction = {"flops_per_step": step_fl, "achieved": step_fl / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
                        "frac": (step_fl / (ms / 1e3) / 1e12 / peak_t) if peak_t else None}
    k_ref = golden_kappa(wl.w, wl.f2, wl.f3)
    kappa_err = float(np.linalg.norm(kappa - k_ref) / np.linalg.norm(k_ref)) if k_ref is not None else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "fcc32-massdis-mesh8: 32-atom LJ fcc (2x2x2 conventional, masses 39.95/83.8 "
                                   "seed 2), 96 modes, 8x8x8 mesh, 260 irreducible q (time reversal), 50 K, "
                                   "Gaussian 0.1 THz",
                       "triplets_per_step_per_gpu": trip,
                       "exchange_pairs": bool(args.pair),
                       "side_stream_sms": side,
                       "velocity_products": "fp32" if args.vel_fp32 else "fp64",
                       "triplets_evaluated_per_step_per_gpu": trip_eval,
                       "triplet_count_note": "value counts every term (irreducible mode, q', nu', nu'') of the "
                                             "linewidth sums; with exchange pairs the kernels contract one q' "
                                             "per unordered {q', q''} with both orderings' weights",
                       "l2": "working set > L2 (W operand 226 MB, "
                       "eigenvector tables 75 MB per step)", "parallelism": f"replicas x{world}"},
            "e2e": {"value": trip_all / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "roofline": roof,
            "step_contraction": step_contraction,
            "kappa_wmk": [kappa[0, 0], kappa[1, 1], kappa[2, 2]],
            "kappa_rel_err_vs_oracle": kappa_err,
            "kappa_error_note": "Frobenius-relative error of this step's RTA kappa against the FP64 oracle's "
                                "(all 260 irreducible q, stored under tests/golden/ with a digest of the inputs)",
            "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if k != "launches" and v[1] > 0},
            "profiled_step_ms": ms_prof}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks

    if args.fp64_q > 0:
        # the FP64 GPU path on a subset of irreducible q: rate and gamma error of this precision
        sub = wl.irr_d[1:1 + args.fp64_q].contiguous()
        g64 = torch.zeros((sub.shape[0], wl.n), dtype=torch.float64, device=device)
        gmx = torch.zeros_like(g64)
        w = wl.w
        wl.ctx.gamma(wl.h, wl.freq, wl.evec, sub, w.temperature, w.shape, w.sigma_thz, w.window, w.f_min_thz,
                     precision="fp64", gamma=g64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wl.ctx.gamma(wl.h, wl.freq, wl.evec, sub, w.temperature, w.shape, w.sigma_thz, w.window, w.f_min_thz,
                     precision="fp64", gamma=g64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        wl.ctx.gamma(wl.h, wl.freq, wl.evec, sub, w.temperature, w.shape, w.sigma_thz, w.window, w.f_min_thz,
                     precision=args.precision, gamma=gmx)
        a, b = gmx.cpu().numpy(), g64.cpu().numpy()
        big = b > 1e-3 * b.max()
        f = wl.freq.cpu().numpy()[wl.irr[1:1 + args.fp64_q]]
        trip64 = int((f >= w.f_min_thz).sum()) * wl.nq * wl.n * wl.n
        line["fp64_path"] = {"value": trip64 / t64, "unit": UNIT, "sample_irreducible_q": int(sub.shape[0]),
                             "gamma_max_rel_err_vs_fp64": float((np.abs(a - b)[big] / b[big]).max())}
        line["speedup_vs_fp64_path"] = value / world / (trip64 / t64)

    if args.kappa_fp64:
        # kappa of each precision against the FP64 GPU path over all irreducible q (the FP64
        # path is parity-tested against the oracle); each run recomputes the whole step
        out = {}
        for prec in ("fp64", "bf16x3", "tf32"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            k = wl.step(prec).copy()
            e1.record(stream)
            torch.cuda.synchronize()
            out[prec] = (k, e0.elapsed_time(e1), wl.g_irr.cpu().numpy().copy())
        k64, _, g64 = out["fp64"]
        big = g64 > 1e-3 * g64.max()
        line["kappa_vs_fp64_path"] = {
            p: {"kappa_rel_err": float(np.linalg.norm(out[p][0] - k64) / np.linalg.norm(k64)),
                "gamma_max_rel_err": float((np.abs(out[p][2] - g64)[big] / g64[big]).max()),
                "step_ms": out[p][1]} for p in ("bf16x3", "tf32")}
        line["kappa_vs_fp64_path"]["fp64_step_ms"] = out["fp64"][1]
        line["kappa_vs_fp64_path"]["kappa_fp64_wmk"] = np.diag(k64).tolist()

    if args.multi_t > 0:
        # several temperatures from one contraction against one call per temperature
        w = wl.w
        temps = [float(x) for x in np.linspace(20.0, 80.0, args.multi_t)]
        gm = torch.zeros((len(temps), wl.irr_d.shape[0], wl.n), dtype=torch.float64, device=device)
        g1 = torch.zeros((wl.irr_d.shape[0], wl.n), dtype=torch.float64, device=device)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        wl.ctx.gamma_multi_t(wl.h, wl.freq, wl.evec, wl.irr_d, temps, w.shape, w.sigma_thz, w.window, w.f_min_thz,
                             precision=args.precision, gamma=gm)
        e1.record(stream)
        for T in temps:
            wl.ctx.gamma(wl.h, wl.freq, wl.evec, wl.irr_d, T, w.shape, w.sigma_thz, w.window, w.f_min_thz,
                         precision=args.precision, gamma=g1)
        e2.record(stream)
        torch.cuda.synchronize()
        ms_m, ms_s = e0.elapsed_time(e1), e1.elapsed_time(e2)
        line["multi_t"] = {"temperatures_K": temps, "ms_one_contraction": ms_m, "ms_one_call_per_T": ms_s,
                           "speedup": ms_s / ms_m,
                           "value": len(temps) * trip / (ms_m / 1e3), "unit": "temperature-triplets/s"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, ctrip, desc = oracle_sample(n_qp=args.cpu_qp)
        line["cpu_baseline"] = {"value": ctrip / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                "sample": desc, "seconds": dt}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Many crystals in one captured graph: the first 16 jobs of the seeded 64-cell sweep (or
    all 64 with --workload batched64).  Prints its own JSON line."""
    import torch
    import paper_2602_23728_gb300 as phx
    import phx_inputs as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = new_context(phx, 0, args)
    n_take = 64 if args.workload == "batched64" else 16
    sweep = P.batched_sweep()[:n_take]
    jobs, trip = [], 0
    t_setup = time.perf_counter()
    for w in sweep:
        c = w.crystal
        f2, f3 = P.ifc_lj_vectorised(c, w.pot)      # same entries as w.ifc2(), w.ifc3(), faster
        n = c.n_modes
        nq = int(np.prod(w.mesh))
        m = w.mesh
        qh = np.array([(i // (m[1] * m[2]) / m[0], (i // m[2]) % m[1] / m[1], i % m[2] / m[2]) for i in range(nq)])
        q = torch.from_numpy(qh).to(dev)
        freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
        evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
        vv = torch.zeros((nq, n, 3, 3), dtype=torch.float64, device=dev)
        ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, freq=freq, evec=evec, vv=vv,
                     want_vel=False)
        irr, f2i, _ = phx.irreducible(w.mesh, w.rotations)
        h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, w.mesh)
        fr = freq.cpu().numpy()
        trip += int((fr[irr] >= w.f_min_thz).sum()) * nq * n * n
        jobs.append(dict(fc3=h, freq=freq, evec=evec, irr=irr, irr_dev=torch.from_numpy(irr.astype(np.int32)).to(dev),
                         T=w.temperature, shape=w.shape, sigma=w.sigma_thz, window=w.window, f_min=w.f_min_thz,
                         gamma=torch.zeros((len(irr), n), dtype=torch.float64, device=dev), vv=vv,
                         full_to_irr=torch.from_numpy(f2i.astype(np.int32)).to(dev),
                         gamma_full=torch.zeros((nq, n), dtype=torch.float64, device=dev),
                         kappa=torch.zeros(9, dtype=torch.float64, device=dev), volume=c.volume))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    t0 = time.perf_counter()
    tuned = ctx.gamma_batched(jobs, precision=args.precision)    # autotune + capture + first run
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.gamma_batched(jobs, precision=args.precision)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    # the same jobs as sequential single-job calls (no graph, default tiles), with the library's
    # per-launch events on: device time per kernel class and per job
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile_enable(True)
    per_job_ms = []
    e0.record(stream)
    for j in jobs:
        j0, j1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        j0.record(stream)
        ctx.gamma(j["fc3"], j["freq"], j["evec"], j["irr_dev"], j["T"], j["shape"], j["sigma"], j["window"],
                  j["f_min"], precision=args.precision, gamma=torch.zeros_like(j["gamma"]))
        j1.record(stream)
        per_job_ms.append((j0, j1))
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    seq_kernel_ms = {k: v[0] for k, v in prof.items() if k != "launches" and v[1] > 0}
    per_job_ms = [a.elapsed_time(b) for a, b in per_job_ms]
    sizes = [(3 * w.crystal.n_atoms, w.mesh[0]) for w in sweep]
    # the FP64 GPU path (same algorithm, FP64 operands) on one irreducible q-point of every job:
    # its rate, and the error of the batched linewidths of that q-point against it
    fp64 = None
    if args.fp64_q > 0:
        t64, trip64, errs = 0.0, 0, []
        for j in jobs:
            k = min(1, len(j["irr"]) - 1)
            sub = j["irr_dev"][k:k + 1].contiguous()
            g64 = torch.zeros((1, j["gamma"].shape[1]), dtype=torch.float64, device=dev)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            ctx.gamma(j["fc3"], j["freq"], j["evec"], sub, j["T"], j["shape"], j["sigma"], j["window"], j["f_min"],
                      precision="fp64", gamma=g64)
            a1.record(stream)
            torch.cuda.synchronize()
            t64 += a0.elapsed_time(a1) / 1e3
            fr = j["freq"].cpu().numpy()
            nqj, nj = fr.shape
            trip64 += int((fr[int(j["irr"][k])] >= j["f_min"]).sum()) * nqj * nj * nj
            ref = g64.cpu().numpy()[0]
            got = j["gamma"][k].cpu().numpy()
            big = ref > 1e-3 * ref.max()
            errs.append(float((np.abs(got - ref)[big] / ref[big]).max()) if big.any() else 0.0)
        fp64 = {"value": trip64 / t64, "unit": UNIT, "sample": "one irreducible q-point per job",
                "gamma_max_rel_err_vs_fp64": max(errs), "per_job_gamma_err": errs}
    line = {"metric": METRIC, "value": trip / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"batched sweep: first {n_take} of 64 seeded mass-disordered LJ fcc cells "
                                   "(seed 3), (modes, mesh edge) = " + json.dumps(sizes),
                       "triplets_per_step": trip, "jobs": n_take},
            "sequential_single_job_calls": {"value": trip / (ms_seq / 1e3), "ms": ms_seq,
                                            "kernel_ms": seq_kernel_ms, "per_job_ms": per_job_ms,
                                            "note": "timed with per-launch events on"},
            "first_call_s_incl_autotune_and_capture": t_first, "setup_s": t_setup,
            "autotuned_q_tile_chain_side_sms": tuned}
    if fp64:
        line["fp64_path"] = fp64
        line["speedup_vs_fp64_path"] = line["value"] / fp64["value"]
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_surrogate(args):
    """4-atom fcc cell, 24^3 mesh at 40 K: exact linewidths on the 8^3 subgrid train the MLP
    ensemble, which fills the dense mesh (q-points outside the network's domain and 5 % more by
    ensemble spread fall back to the exact kernel).  The value is the dense mesh's
    exact-equivalent triplets divided by the surrogate pipeline's time (the run of median time
    among independent trainings); the exact dense run and the coarse-mesh conductivity are
    reported beside it."""
    import torch
    import paper_2602_23728_gb300 as phx
    import phx_inputs as P
    from paper_2602_23728_gb300 import surrogate
    torch.cuda.set_device(0)
    ctx = new_context(phx, 0, args)
    w = P.fcc_conventional_4(mesh=(24, 24, 24), temperature=40.0)
    c = w.crystal
    f2, f3 = w.ifc2(), w.ifc3()
    runs = []
    # every timed run is an independent training (seeds 1, 2, ...): one training is one draw of
    # the seeded splits and initial weights, so times and errors are reported as medians
    for k in range(max(args.steps, 1) + 1):          # the first run (seed 0) warms up
        r = surrogate.run(ctx, phx, c.lattice, c.masses, f2.idx, f2.val, f3.idx, f3.val, w.mesh, 3, w.rotations,
                          w.temperature, precision=args.precision, seed=k)
        if k > 0:
            runs.append(r)

    def t_pipeline(r):
        t = r["timings"]
        return t["exact_subgrid"] + t["features"] + t["train"] + t["infer"] + t["fallback"]
    order = np.argsort([t_pipeline(x) for x in runs])
    r = runs[order[len(order) // 2]]                 # the run of median pipeline time
    t = r["timings"]
    t_sur = t_pipeline(r)
    errs = [x["kappa_rel_err_surrogate"] for x in runs]
    line = {"metric": METRIC, "value": r["triplets_exact"] / t_sur, "unit": UNIT, "n_gpus": 1, "steps": len(runs),
            "warmup": 1, "ms_per_step": 1e3 * t_sur, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "surrogate: 4-atom conventional LJ fcc, 24^3 mesh (455 irreducible q), 40 K; "
                                   "MLP 4-128-128-128-1 x4 trained on the 8^3 subgrid (35 irreducible q)",
                       "exact_equivalent_triplets": r["triplets_exact"]},
            "exact_dense_path": {"value": r["triplets_exact"] / t["exact_full"], "s": t["exact_full"]},
            "kappa_rel_err": {"surrogate_median": float(np.median(errs)), "surrogate_per_run": errs,
                              "coarse_mesh_exact": r["kappa_rel_err_coarse"],
                              "nearest_subgrid_interpolation": r["kappa_rel_err_interp"]},
            "heldout_rel_err": {"median": r["heldout_median_rel_err"], "max": r["heldout_max_rel_err"]},
            "timings_s": t, "n_fallback_q": r["n_fallback_q"], "n_outside_q": r["n_outside_q"], "n_irr": r["n_irr"],
            "final_loss": list(map(float, r["final_loss"])), "epochs_run": r["epochs_run"]}
    print(json.dumps(line, default=float), flush=True)
    ctx.close()
    return 0


def run_cell(args):
    """Gamma-only disordered cell: 1000 atoms (3000 modes), Lorentzian (half width 0.05 THz),
    300 K.  One step = the 3000 x 3000 FP64 eigensolve, the linewidths of all modes and the
    QHGK conductivity (Eq. qhgk).  A
    triplet is one (lambda, nu', nu'') with lambda above f_min, so a step holds
    n_live x 3000^2 of them (each unordered triple is evaluated once; the count is that of the
    ordered sum).  The FP64 GPU path is timed once beside it and the oracle on two modes."""
    import torch
    import paper_2602_23728_gb300 as phx
    import phx_inputs as P
    import oracle as O
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = new_context(phx, 0, args)
    t_setup = time.perf_counter()
    w = P.gamma_disordered_1000(reps=(args.cell_reps,) * 3)
    c = w.crystal
    f2, f3 = P.ifc_lj_vectorised(c, w.pot)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, (1, 1, 1))
    n = c.n_modes
    q = torch.zeros((1, 3), dtype=torch.float64, device=dev)
    freq = torch.zeros((1, n), dtype=torch.float64, device=dev)
    evec = torch.zeros((1, n, n), dtype=torch.complex128, device=dev)
    gam = torch.zeros(n, dtype=torch.float64, device=dev)
    kw = dict(shape=w.shape, sigma=w.sigma_thz, window=w.window, f_min=w.f_min_thz)
    t_setup = time.perf_counter() - t_setup

    f2v = f2.val.reshape(-1, 9)

    def step(prec):
        ctx.harmonic(c.lattice, c.masses, f2.idx, f2v, q, freq=freq, evec=evec, want_vel=False, want_vv=False)
        ctx.gamma_cell(h, freq[0], evec[0], w.temperature, precision=prec, gamma=gam, **kw)
        return ctx.kappa_qhgk(c.lattice, c.masses, c.positions, f2.idx, f2v, freq[0], evec[0], gam, w.temperature,
                              f_min=w.f_min_thz)

    for _ in range(args.warmup):
        step(args.precision)
    torch.cuda.synchronize()
    n_live = int((freq[0] >= w.f_min_thz).sum().item())
    trip = n_live * n * n
    stream = torch.cuda.current_stream()
    ctx.profile_enable(False)            # no per-launch events in the timed loop; zeroes the launch count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step(args.precision)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = ctx.profile_read()["launches"]
    ctx.profile_enable(True)             # one separate step with events around every launch
    kappa_q = step(args.precision)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    g_mixed = gam.cpu().numpy().copy()
    f_h = freq[0].cpu().numpy()
    e_h = evec[0].cpu().numpy()
    # FP64 GPU path (same algorithm, FP64 operands and CUDA-core GEMM), timed once
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.gamma_cell(h, freq[0], evec[0], w.temperature, precision="fp64", gamma=gam, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    g64 = gam.cpu().numpy()
    big = g64 > 1e-3 * g64.max()
    rel = float((np.abs(g_mixed - g64)[big] / g64[big]).max())
    peaks, peak_src = load_peaks()
    per = {k: v for k, v in prof.items() if k != "launches" and v[1] > 0}
    ms_k = {k: v[0] for k, v in per.items()}
    top = max(("cell_sparse", "cell_gemm", "cell_transpose"), key=lambda k: ms_k.get(k, 0.0))
    ms_top, n_top, fl_top, by_top = per[top]
    if top == "cell_gemm":
        peak = peaks["bf16_tflops_sustained"] / 3.0 if args.precision == "bf16x3" else \
            peaks["bf16_tflops_sustained"] * NOMINAL_TF32_OVER_BF16
        ach = fl_top / (ms_top / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "sym_tc_kernel", "peak_note": f"of {peak_src} bf16 sustained"
                + (" / 3 (three bf16 MMAs per product)" if args.precision == "bf16x3" else " x nominal tf32/bf16")}
    elif top == "cell_sparse":
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = fl_top / (ms_top / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": None, "kernel": "xform_kernel",
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}
    else:
        ach = by_top / (ms_top / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": top}
    # the conductivity with the FP64 linewidths, for the kappa error of the chosen precision
    kappa_64 = ctx.kappa_qhgk(c.lattice, c.masses, c.positions, f2.idx, f2v, freq[0], evec[0], gam, w.temperature,
                              f_min=w.f_min_thz)
    kerr = float(np.linalg.norm(kappa_q - kappa_64) / np.linalg.norm(kappa_64))
    line = {"metric": METRIC, "value": trip / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "kappa_qhgk_wmk": np.diag(kappa_q).tolist(), "kappa_rel_err_vs_fp64_linewidths": kerr,
            "config": {"workload": "Gamma-only disordered cell: 10x10x10 primitive LJ fcc = 1000 atoms, 3000 modes, "
                                   "N(0, 0.05 A) noise seed 5 relaxed to max force 1e-8 eV/A, 50/50 masses "
                                   "39.95/83.8, sparse COO Phi3 (r_c 8.5 A), Lorentzian half width 0.05 THz, 300 K",
                       "triplets_per_step": trip, "modes_above_f_min": n_live,
                       "inputs_vs_l2": "eigenvectors 72 MB FP64 (hi/lo operand copies 36 MB) + per-chunk operands "
                                       "of several GB: each step streams well over the 129 MB L2"},
            "roofline": roof,
            "fp64_gpu_path": {"value": trip / (ms64 / 1e3), "ms": ms64, "gamma_rel_err_vs_fp64": rel},
            "kernel_ms_per_step": ms_k, "gpu_launches": int(launches), "setup_s": t_setup}
    if not args.no_cpu_baseline:
        modes = [int(np.nonzero(f_h >= 0.5)[0][0]), int(np.argmax(f_h > 1.0))]
        t0 = time.perf_counter()
        O.gammapoint.gamma_modes(f3.idx, f3.val, c.masses, f_h, e_h.real, modes, w.temperature, w.shape, w.sigma_thz)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(modes) * n * n / dt, "unit": UNIT, "cores": blas_threads(),
                                "kind": "oracle", "sample": f"oracle per-mode linewidths of {len(modes)} of the "
                                f"{n_live} modes (all {n}^2 partner pairs each), eigenvectors shared"}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    print(json.dumps(line, default=float), flush=True)
    ctx.close()
    return 0


def run_sc(args):
    """Iterative BTE on the fcc32 workload (Eqs. gamma1, sc_iter): one step = harmonic phonons
    with velocities on the 8x8x8 mesh, one contraction giving Gamma0 and the folded Gamma1
    (24,960 x 24,960, FP32 on the device for the tensor-core precisions) of the 260
    time-reversal representatives, then the iteration to a relative change of Tr(kappa)/3
    below --sc-tol.  Throughput counts the contraction's triplets, as the headline does."""
    import torch
    import paper_2602_23728_gb300 as phx
    import oracle as O
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = new_context(phx, 0, args)
    ctx.set_option("sc_matrix_free", args.sc_matrix_free)
    wl = Workload(phx, ctx, args.precision, dev, mesh=(args.sc_mesh,) * 3)
    w, c = wl.w, wl.c
    n, nq = wl.n, wl.nq
    n_tr = len(wl.irr)
    R = n_tr * n
    vel = torch.zeros((nq, n, 3), dtype=torch.float64, device=dev)
    g0 = torch.zeros((n_tr, n), dtype=torch.float64, device=dev)
    mfp = torch.zeros((n_tr, n, 3), dtype=torch.float64, device=dev)
    kw = dict(shape=w.shape, sigma=w.sigma_thz, window=w.window, f_min=w.f_min_thz, max_iter=args.sc_iter,
              tol=args.sc_tol)

    def step(prec):
        ctx.harmonic(c.lattice, c.masses, wl.f2.idx, wl.f2val, wl.q, freq=wl.freq, evec=wl.evec, vel=vel,
                     want_vv=False)
        return ctx.kappa_sc(c.lattice, c.masses, wl.h, wl.freq, wl.evec, vel, w.temperature, precision=prec,
                            gamma0=g0, mfp=mfp, **kw)

    for _ in range(args.warmup):
        r = step(args.precision)
    torch.cuda.synchronize()
    trip = wl.triplets()
    stream = torch.cuda.current_stream()
    ctx.profile_enable(False)            # no per-launch events in the timed loop; zeroes the launch count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            r = step(args.precision)
            iters.append(r["n_iter"])
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = ctx.profile_read()["launches"]
    ctx.profile_enable(True)             # one separate step with events around every launch
    r = step(args.precision)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    peaks, peak_src = load_peaks()
    per = {k: v for k, v in prof.items() if k != "launches" and v[1] > 0}
    ms_k = {k: v[0] for k, v in per.items()}
    kappa = r["kappa"]
    line = {"metric": METRIC, "value": trip / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "kappa_rta_wmk": float(np.trace(kappa[0]) / 3), "kappa_sc_wmk": float(np.trace(kappa[-1]) / 3),
            "kappa_sc_diag_wmk": np.diag(kappa[-1]).tolist(), "iterations": iters, "converged": r["converged"],
            "config": {"workload": "fcc32-massdis-mesh%d iterative BTE: 32-atom LJ fcc (masses 39.95/83.8 seed 2), "
                                   "96 modes, %dx%dx%d, 50 K, Gauss 0.1 THz; Gamma1 over the %d time-reversal "
                                   "representatives (R = %d rows)" % ((args.sc_mesh,) * 4 + (n_tr, R)),
                       "triplets_per_step": trip, "sc_tol": args.sc_tol, "sc_max_iter": args.sc_iter,
                       "gamma1_form": "matrix-free (applied in every iteration's contraction pass)"
                       if args.sc_matrix_free == 1 else "dense, resident in HBM (matrix-free if it did not fit)",
                       "gamma1_bytes": R * ((R + 127) // 128 * 128) * (8 if args.precision == "fp64" else 4),
                       "inputs_vs_l2": "Gamma1 (2.5 GB FP32) and the contraction operands stream well over the "
                                       "129 MB L2 every pass"},
            "kernel_ms_per_step": ms_k, "gpu_launches": int(launches)}
    if "sc_step" in per:
        ms_s, n_s, fl_s, by_s = per["sc_step"]
        ach = by_s / (ms_s / 1e3) / 1e9
        line["sc_step_roofline"] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                    "frac": ach / peaks["hbm_gbs"], "launches": n_s, "traffic": None,
                                    "kernel": "sc_step_kernel",
                                    "peak_note": f"of {peak_src} copy bandwidth"}
    line["roofline"] = roofline_of(prof, 1, ms, args.precision, peaks, peak_src, "fcc32-sc")
    if args.kappa_fp64:
        # the same BTE step with every contraction in FP64 (and once in TF32): the kappa error of
        # each precision, RTA iterate and converged iterate
        ref = {}
        for prec in ("fp64", "tf32"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rr = step(prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ref[prec] = (rr["kappa"], e0.elapsed_time(e1), rr["n_iter"])
        k64 = ref["fp64"][0]
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        line["kappa_vs_fp64_path"] = {
            "fp64_step_ms": ref["fp64"][1], "kappa_sc_fp64_wmk": float(np.trace(k64[-1]) / 3),
            "fp64_iterations": ref["fp64"][2],
            args.precision: {"kappa_rta_rel_err": rel(kappa[0], k64[0]), "kappa_sc_rel_err": rel(kappa[-1], k64[-1])},
            "tf32": {"kappa_rta_rel_err": rel(ref["tf32"][0][0], k64[0]),
                     "kappa_sc_rel_err": rel(ref["tf32"][0][-1], k64[-1]), "step_ms": ref["tf32"][1]}}
    if not args.no_cpu_baseline:
        # the oracle's scattering rows of one representative over a bounded q' sample
        f = wl.freq.cpu().numpy()
        e = wl.evec.cpu().numpy()
        f3 = w.ifc3()
        fc3o = O.anharmonic.FC3(f3.idx, f3.val, c.masses)
        n_qp = args.cpu_qp or 48
        kint = O.grid.mesh_int(w.mesh)
        qred = O.grid.mesh_qred(w.mesh)
        iq = int(wl.irr[1])
        nocc = O.occupation.bose(f, w.temperature)
        t0 = time.perf_counter()
        for iqp in range(n_qp):
            iqpp = int(O.grid.mesh_index(-(kint[iq] + kint[iqp]), w.mesh))
            V = O.anharmonic.v3(fc3o, e[iq], qred[iqp], e[iqp], -(qred[iq] + qred[iqp]), e[iqpp])
            W = O.anharmonic.pair_weights(f[iq], f[iqp], f[iqpp], nocc[iqp], nocc[iqpp], w.shape, w.sigma_thz,
                                          w.f_min_thz, w.window)
            x = np.abs(V) ** 2 * W
            g_part, cols_q1, cols_q2 = x.sum(axis=(1, 2)), x.sum(axis=2), x.sum(axis=1)
        dt = time.perf_counter() - t0
        valid = int((f[iq] >= w.f_min_thz).sum())
        line["cpu_baseline"] = {"value": valid * n_qp * n * n / dt, "unit": UNIT, "cores": blas_threads(),
                                "kind": "oracle", "sample": f"oracle Gamma0 and Gamma1 rows of representative {iq} "
                                f"over {n_qp} of {nq} q' (the iteration itself not included)"}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    print(json.dumps(line, default=float), flush=True)
    ctx.close()
    return 0


def run_sc64(args):
    """Iterative BTE on a 64-atom cell (4x4x4 primitive LJ fcc, 50/50 masses 39.95/83.8 seed 11,
    192 modes) on a 12x12x12 mesh at 50 K, Gaussian 0.1 THz: 868 time-reversal representatives,
    Gamma1 of 166,656 x 166,656 in FP32 (111 GB) held on the device.  One step, as fcc32-sc."""
    import torch
    import paper_2602_23728_gb300 as phx
    import phx_inputs as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = new_context(phx, 0, args)
    c = P.random_masses(P.fcc_primitive_multiple(5.26, (4, 4, 4)), 39.95, 83.8, seed=11)
    mesh = (12, 12, 12)
    f2, f3 = P.ifc_lj_vectorised(c, P.LennardJones())
    nq, n = int(np.prod(mesh)), c.n_modes
    qh = np.array([(i // (mesh[1] * mesh[2]) / mesh[0], (i // mesh[2]) % mesh[1] / mesh[1], i % mesh[2] / mesh[2])
                   for i in range(nq)])
    q = torch.from_numpy(qh).to(dev)
    freq = torch.zeros((nq, n), dtype=torch.float64, device=dev)
    evec = torch.zeros((nq, n, n), dtype=torch.complex128, device=dev)
    vel = torch.zeros((nq, n, 3), dtype=torch.float64, device=dev)
    h = ctx.fc3(c.lattice, c.masses, f3.idx, f3.val, mesh)
    n_tr = phx.time_reversal_count(mesh)
    g0 = torch.zeros((n_tr, n), dtype=torch.float64, device=dev)
    mfp = torch.zeros((n_tr, n, 3), dtype=torch.float64, device=dev)

    def step():
        ctx.harmonic(c.lattice, c.masses, f2.idx, f2.val.reshape(-1, 9), q, freq=freq, evec=evec, vel=vel,
                     want_vv=False)
        return ctx.kappa_sc(c.lattice, c.masses, h, freq, evec, vel, 50.0, shape="gauss", sigma=0.1, window=2.0,
                            f_min=0.01, max_iter=args.sc_iter, tol=args.sc_tol, precision=args.precision,
                            gamma0=g0, mfp=mfp)

    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        r = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    fr = freq.cpu().numpy()
    irr_tr = np.unique([min(i, int(O_neg)) for i, O_neg in enumerate(_neg_index(mesh))])
    trip = int((fr[irr_tr] >= 0.01).sum()) * nq * n * n
    R = n_tr * n
    line = {"metric": METRIC, "value": trip / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "cell64-mesh12 iterative BTE: 64-atom LJ fcc (4x4x4 primitive, masses 39.95/83.8 "
                                   "seed 11), 192 modes, 12x12x12, 50 K, Gauss 0.1 THz; Gamma1 over the %d "
                                   "time-reversal representatives (R = %d rows, %.0f GB in FP32)"
                                   % (n_tr, R, R * ((R + 127) // 128 * 128) * 4 / 1e9),
                       "triplets_per_step": trip},
            "kappa_rta_wmk": float(np.trace(r["kappa"][0]) / 3), "kappa_sc_wmk": float(np.trace(r["kappa"][-1]) / 3),
            "iterations": r["n_iter"], "converged": r["converged"]}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    print(json.dumps(line, default=float), flush=True)
    ctx.close()
    return 0


def _neg_index(mesh):
    m1, m2, m3 = mesh
    out = []
    for i in range(m1 * m2 * m3):
        a, b, c = i // (m2 * m3), (i // m3) % m2, i % m3
        out.append((((m1 - a) % m1) * m2 + (m2 - b) % m2) * m3 + (m3 - c) % m3)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="phx", choices=["phx", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32", "fp64"])
    ap.add_argument("--fp64-q", type=int, default=4, help="irreducible q timed on the FP64 GPU path (0: skip)")
    ap.add_argument("--cpu-qp", type=int, default=None, help="q' of the oracle sample (default all)")
    ap.add_argument("--kappa-fp64", action="store_true",
                    help="also run the whole step in FP64 and TF32 and report the kappa error of each precision")
    ap.add_argument("--multi-t", type=int, default=4,
                    help="temperatures timed in one contraction vs one call each (0: skip)")
    ap.add_argument("--ref-qp", type=int, default=64, help="q' per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="fcc32",
                    choices=["fcc32", "fcc32-sc", "sc64-mesh12", "batched16", "batched64", "surrogate24", "cell1000"],
                    help="fcc32: the headline workload; batched16/64: the many-crystal sweep; surrogate24: the "
                         "learned-linewidth pipeline; cell1000: the Gamma-only 1000-atom disordered cell "
                         "(each its own JSON line); fcc32-sc: the iterative BTE on the headline crystal")
    ap.add_argument("--sc-iter", type=int, default=100, help="fcc32-sc: maximum iterations")
    ap.add_argument("--sc-matrix-free", type=int, default=0, choices=[0, 1, 2],
                    help="fcc32-sc: Gamma1 dense when it fits (0), always matrix-free (1), always dense (2)")
    ap.add_argument("--sc-tol", type=float, default=1e-6, help="fcc32-sc: relative change of Tr(kappa)/3")
    ap.add_argument("--sc-mesh", type=int, default=8,
                    help="fcc32-sc: mesh edge (8 = the bench size; 4 keeps the per-launch shape of the "
                         "contraction for profiler captures)")
    ap.add_argument("--cell-reps", type=int, default=10,
                    help="cell1000: primitive cells per edge of the disordered cell (10 = the 1000-atom "
                         "workload; 6 = a 216-atom cell of the same kind for profiler captures)")
    ap.add_argument("--pair", type=int, default=1, choices=[0, 1],
                    help="1: the tensor-core passes evaluate each exchange pair {q', q''} once (default); "
                         "0: every q' of the mesh")
    ap.add_argument("--vel-fp32", type=int, default=1, choices=[0, 1],
                    help="1: velocity products of the harmonic step with FP32 products and sums (default; the "
                         "eigensolve, occupations and the kappa sum stay FP64); 0: FP64")
    ap.add_argument("--irr-limit", type=int, default=0,
                    help="profiling aid: process only the first N irreducible q per step (0: all)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched16", "batched64"):
        return run_batched(args)
    if args.workload == "surrogate24":
        return run_surrogate(args)
    if args.workload == "cell1000":
        return run_cell(args)
    if args.workload == "fcc32-sc":
        return run_sc(args)
    if args.workload == "sc64-mesh12":
        return run_sc64(args)
    return run_phx(args)


if __name__ == "__main__":
    sys.exit(main())
