"""Host-side logic that needs no GPU: the exchange-pair count the bench reports (against a
brute-force count over the mesh), the bench's roofline arithmetic and its source-keyed DRAM
traffic lookup, and the surrogate workflow's choice of the q-points sent back to the exact
kernel."""
import math
import os

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("mesh", [(3, 4, 5), (4, 4, 4), (2, 3, 2), (6, 1, 1), (8, 8, 8)])
def test_pair_count_is_the_unordered_pair_count(bench, mesh):
    """One q' per unordered partner pair {q', q'' = -(q + q')}: the number of mesh points q'
    with index(q') <= index(q''), for every q of the mesh."""
    nq = int(np.prod(mesh))
    qs = range(nq) if nq <= 64 else range(0, nq, 37)
    for iq in qs:
        brute = sum(1 for qp in range(nq) if qp <= O.grid.third_index(iq, qp, mesh))
        assert bench.pair_count(iq, mesh, True) == brute, (mesh, iq)
        assert bench.pair_count(iq, mesh, False) == nq


def test_roofline_arithmetic(bench):
    """frac = algorithmic flops / event time / tensor peak of the precision (BF16x3: sustained
    bf16 / 3), the HBM figure beside it, and the SM-share variant for a class confined to part
    of the GPU; a class off the tensor list is reported against the copy bandwidth."""
    peaks = {"hbm_gbs": 6801.7, "bf16_tflops": 1909.0, "bf16_tflops_sustained": 1704.9}
    nl, fl1, by1 = 556, 1.63e11, 8.49e8
    prof = {"chain": (336.0, nl, nl * fl1, nl * by1), "dft": (270.0, nl, nl * 1e10, nl * 2e9),
            "fold": (55.0, 260, 1e9, 260 * 2.26e8), "launches": 12000}
    r = bench.roofline_of(prof, 1, 378.0, "bf16x3", peaks, "measured", "none", sm_share={"chain": (104, 152)})
    ach = nl * fl1 / 0.336 / 1e12
    assert r["kernel"] == "chain" and r["bound"] == "tensor"
    assert math.isclose(r["achieved"], ach, rel_tol=1e-12)
    assert math.isclose(r["frac"], ach / (1704.9 / 3), rel_tol=1e-12)
    assert math.isclose(r["frac_of_its_sms_peak"], r["frac"] * 152 / 104, rel_tol=1e-12)
    assert math.isclose(r["hbm"]["frac"], nl * by1 / 0.336 / 1e9 / 6801.7, rel_tol=1e-12)
    assert math.isclose(r["share_of_step"], 336.0 / 378.0, rel_tol=1e-12)
    assert r["traffic"] is None                               # no capture for workload "none"
    r32 = bench.roofline_of(prof, 1, 378.0, "tf32", peaks, "measured", "none")
    assert math.isclose(r32["frac"], ach / (1704.9 * 1.1 / 2.25), rel_tol=1e-12)
    only_fold = {"fold": prof["fold"], "launches": 1}
    rf = bench.roofline_of(only_fold, 1, 378.0, "bf16x3", peaks, "measured", "none")
    assert rf["bound"] == "hbm" and math.isclose(rf["frac"], 260 * 2.26e8 / 0.055 / 1e9 / 6801.7, rel_tol=1e-12)


def test_traffic_lookup_is_keyed_by_source_hash(bench, tmp_path, monkeypatch):
    """A stored DRAM figure is reported only while the hash of the kernel sources matches the
    one recorded with the capture."""
    h = bench.kernel_source_hash()
    f = tmp_path / "traffic.txt"
    f.write_text(f"# comment\nfcc32 chain bf16x3 123456 {h}\nfcc32 dft bf16x3 999 0000000000000000\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("chain", "bf16x3", "fcc32") == 123456.0
    assert bench.measured_traffic("dft", "bf16x3", "fcc32") is None        # stale hash
    assert bench.measured_traffic("chain", "tf32", "fcc32") is None


def test_fallback_rows():
    """Every out-of-domain q-point (infinite score) goes to the exact kernel, plus the
    ceil((100 - pct) % of all candidates) largest finite spreads; ties keep candidate order."""
    from paper_2602_23728_gb300.surrogate import fallback_rows
    rng = np.random.default_rng(5)
    score = rng.uniform(0.0, 1.0, 200)
    score[[3, 17, 150]] = np.inf
    score[[40, 41]] = 5.0                                    # a tie at the top of the finite ones
    cand = np.array([k for k in range(200) if k % 7 != 0])   # candidates: not on the subgrid
    ood, pick = fallback_rows(score, cand, 95.0)
    assert sorted(ood.tolist()) == [3, 17, 150]
    n_fb = math.ceil(0.05 * len(cand))
    assert len(pick) == n_fb and not np.isinf(score[pick]).any()
    assert pick[0] == 40 and pick[1] == 41
    finite = [k for k in cand if np.isfinite(score[k])]
    top = sorted(finite, key=lambda k: -score[k])[:n_fb]
    assert sorted(pick.tolist()) == sorted(top)
    ood0, pick0 = fallback_rows(score, cand, 100.0)
    assert len(pick0) == 0 and len(ood0) == 3


def test_subgrid_points():
    from paper_2602_23728_gb300.surrogate import subgrid_points
    mesh = (6, 4, 8)
    pts = subgrid_points(mesh, 2)
    assert len(pts) == 3 * 2 * 4
    for p in pts:
        i, j, k = p // (mesh[1] * mesh[2]), (p // mesh[2]) % mesh[1], p % mesh[2]
        assert i % 2 == 0 and j % 2 == 0 and k % 2 == 0


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host's cores, a bounded q' sample per
    step) prints one JSON line with the metric, unit and direction of the GPU arm and its
    cpu_baseline and e2e objects."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-qp", "4"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "triplets/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
