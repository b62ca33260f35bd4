"""Batching (waves of several circuits in one set of launches) and serving (request loop with
admission by projected device memory and continuous batching), through the C ABI.

Each circuit's result in the mix must be the one it gets alone: identical bond dimensions,
unswap logs, layouts and peak bitstrings, and gauge-invariant values within the path's
tolerance (FP64: spectra 1e-10, p_peak 1e-12; mixed precision: 1e-6).  Every kernel of the
factorisation computes a task in an order that does not depend on the other tasks of its
launch (the Jacobi sums each inner product in an order fixed by the row length, whatever group
width the launch takes), so an FP64 circuit's spectra and p_peak are also bit-identical alone
and in the mix."""
import time

import numpy as np
import pytest

from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}     # precision -> (spectra, p_peak)


def mix():
    """Circuits of different sizes, perturbations and configurations."""
    return [
        (W.hidden_permutation_mirror(8, 20, 0.02, seed=1), dict(eps=1e-10, chi_max=64, tau=600)),
        (W.hidden_permutation_mirror(10, 24, 0.0, seed=2), dict(eps=1e-10, chi_max=64, tau=800)),
        (W.hidden_permutation_mirror(9, 18, 0.03, seed=3), dict(eps=1e-10, chi_max=32, tau=500)),
        (W.hidden_permutation_mirror(8, 20, 0.02, seed=4),
         dict(eps=1e-5, chi_max=64, tau=600, precision=binding.PRECISION_TF32X3)),
        (W.workload_line12(5), dict(eps=1e-12, chi_max=64, tau=1e6)),
    ]


def summary(c, n):
    bits, p, _ = c.extract_peak()
    return {"chi": list(c.bond_dims()), "log": c.unswap_log().tolist(), "lay": [x.tolist() for x in c.layouts()],
            "spec": [c.spectrum(b) for b in range(n - 1)], "bits": bits, "p": p}


def alone(circ, kw):
    ctx = binding.Context(**kw)
    c = ctx.load_circuit(circ)
    st = c.contract()
    out = summary(c, circ.n_qubits)
    out["n_waves"] = st["n_waves"]
    c.close()
    ctx.close()
    return out


def same(a, b, prec):
    tol_s, tol_p = TOL[prec]
    assert a["chi"] == b["chi"]
    assert a["log"] == b["log"]
    assert a["lay"] == b["lay"]
    assert np.array_equal(a["bits"], b["bits"])
    assert abs(a["p"] - b["p"]) <= tol_p
    for x, y in zip(a["spec"], b["spec"]):
        assert np.max(np.abs(x - y)) <= tol_s
    if prec == 0:
        assert a["p"] == b["p"]
        for x, y in zip(a["spec"], b["spec"]):
            assert np.array_equal(x, y)


def test_batch_contract_matches_alone():
    cases = mix()
    ref = [alone(circ, kw) for circ, kw in cases]
    ctxs = [binding.Context(**kw) for _, kw in cases]
    circs = [ctx.load_circuit(circ) for ctx, (circ, _) in zip(ctxs, cases)]
    batch = binding.Batch(ctxs[0], max_tasks=128)
    statuses, stats = batch.contract(circs)
    assert all(s >= 0 for s in statuses)
    for (circ, kw), c, r in zip(cases, circs, ref):
        same(summary(c, circ.n_qubits), r, kw.get("precision", 0))
    cnt = batch.counters()
    # the waves of different circuits really shared launches
    assert cnt["launches"] < sum(s["n_waves"] for s in stats)
    assert cnt["max_tasks"] > max(circ.n_qubits // 2 for circ, _ in cases)
    for c in circs:
        c.close()
    batch.close()
    for ctx in ctxs:
        ctx.close()


def test_server_continuous_batching_results_match_alone():
    cases = mix()
    ref = [alone(circ, kw) for circ, kw in cases]
    srv = binding.Server(max_resident=3, memory_budget=32 << 30, max_tasks=128)
    tickets = []
    # three at once, the rest while those are on the GPU
    for circ, kw in cases[:3]:
        tickets.append(srv.submit(circ, n_samples=50, seed=9, **kw))
    time.sleep(0.05)
    for circ, kw in cases[3:]:
        tickets.append(srv.submit(circ, n_samples=50, seed=9, **kw))
    for t, (circ, kw), r in zip(tickets, cases, ref):
        res, bits, samples = srv.wait(t, timeout_s=600)
        assert res["status"] == 0
        assert np.array_equal(bits, r["bits"])
        assert abs(res["p_peak"] - r["p"]) <= TOL[kw.get("precision", 0)][1]
        if kw.get("precision", 0) == 0:
            assert res["p_peak"] == r["p"]
        assert samples.shape == (50, circ.n_qubits)
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
    st = srv.stats()
    assert st["completed"] == len(cases) and st["failed"] == 0
    assert 1 <= st["max_resident_seen"] <= 3
    assert 0 < st["p50_s"] <= st["p99_s"]
    assert st["circuits_per_hour"] > 0
    assert st["launches"] < sum(r["n_waves"] for r in ref)
    srv.close()


def test_server_admission_by_projected_memory():
    circ = W.hidden_permutation_mirror(8, 16, 0.02, seed=6)
    kw = dict(eps=1e-10, chi_max=64, tau=500)
    one = binding.projected_bytes(8, 64, 0)
    assert one > 0
    # room for one resident circuit at a time, three slots
    srv = binding.Server(max_resident=3, memory_budget=int(1.5 * one), max_tasks=64)
    tickets = [srv.submit(circ, **kw) for _ in range(3)]
    # too large for the budget even alone
    big = W.hidden_permutation_mirror(12, 8, 0.0, seed=7)
    t_big = srv.submit(big, eps=1e-10, chi_max=1024, tau=1e6)
    bits0 = None
    for t in tickets:
        res, bits, _ = srv.wait(t, timeout_s=600)
        assert res["status"] == 0
        bits0 = bits if bits0 is None else bits0
        assert np.array_equal(bits, bits0)
    res, _, _ = srv.wait(t_big, timeout_s=600)
    assert res["status"] == -3          # PC_ERR_OOM: never admitted
    st = srv.stats()
    assert st["max_resident_seen"] == 1
    assert st["max_bytes_seen"] <= int(1.5 * one)
    assert st["failed"] == 1 and st["completed"] == 3
    srv.close()
