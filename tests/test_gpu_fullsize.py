"""Parity in the benchmark's own configuration: 28 qubits, the saturated MPO with every interior
bond at chi = 256 (1024 x 1024 bond matrices), eps = 1e-10, chi_max = 256.  The oracle routes and
absorbs the first gate of the benchmark step's layer (eight routing SWAPs and the gate, nine
factorisations at the chi_max cap, each with a relative gap of ~2e-3 at the cap so the kept
subspace is well defined); the library applies the same nine operators through the C ABI.
Compared: every bond dimension, every bond spectrum (1e-10), and the amplitudes <x|M|0> of
eight bitstrings (1e-10 of the largest) — quantities that do not depend on the gauge of the
site tensors."""
import numpy as np
import pytest

from oracle import mpo
from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, CHI, EPS, CURSOR = 28, 256, 1e-10, 12


def test_bench_configuration_first_gate_matches_oracle():
    circ = W.workload_unswap28(0)
    B, lam = W.peaked_saturated_state(N, CHI, 0)
    cfg = mpo.Config(eps=EPS, chi_max=CHI, tau=1e6)
    ctr = mpo.Contraction(circ, cfg)
    ctr.state.B = [b.copy() for b in B]
    ctr.state.lam = [l.copy() for l in lam]
    ops = []
    update = ctr.state.apply

    def recorded(j, u16, c):
        ops.append((j, np.array(u16)))
        return update(j, u16, c)

    ctr.state.apply = recorded
    ctr._route_and_apply(mpo.SIDE_LEFT, ctr.left_layers[CURSOR][0])
    assert len(ops) == 9

    ctx = binding.Context(eps=EPS, chi_max=CHI, tau=1e6)
    c = ctx.load_gates(N, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    c.set_state(B, lam)
    for j, u16 in ops:
        c.apply_updates([j], u16[None])
    # the chi = 256 interior updates ran with the deflated FP64 sweeps (exactness is checked
    # by the library after the sweeps; the comparisons below check the results)
    assert c.stats()["n_deflated"] >= 1

    assert list(c.bond_dims()) == ctr.state.bond_dims()
    for bond in range(N - 1):
        np.testing.assert_allclose(c.spectrum(bond), ctr.state.lam[bond], atol=1e-10, rtol=0)
    # amplitudes of M|0> with the layouts the library holds (identity: pc_apply_updates routes nothing)
    out = mpo.project_zero(mpo.Result(ctr.state, mpo.Layout(N), mpo.Layout(N)))
    rng = np.random.default_rng(4)
    xs = np.vstack([np.zeros((1, N), np.uint8), rng.integers(0, 2, (7, N)).astype(np.uint8)])
    ref = mpo.amplitudes(out, xs)
    got = c.amplitudes(xs)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    c.close()
    ctx.close()


def test_unswap_stage_certificate_matches_full_trials_and_oracle():
    """One parallel unswap stage (App. A.1) on the saturated 28-qubit state, its trials decided
    by the lower-bound certificate and, separately, by full factorisations: identical unswap
    logs, bond dimensions and spectra (1e-10).  The decisions of the first batch (SWAPs from
    both sides on the even bonds) equal the oracle's full-SVD counts against chi_old."""
    B, lam = W.peaked_saturated_state(N, CHI, 0)
    res = {}
    for certify in (1, 0):
        ctx = binding.Context(eps=EPS, chi_max=CHI, tau=1e6, certify_trials=certify)
        c = ctx.load_gates(N, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
        c.set_state(B, lam)
        c.unswap()
        res[certify] = (list(c.unswap_log().tolist()), list(c.bond_dims()),
                        [c.spectrum(b) for b in range(N - 1)], c.stats())
        c.close()
        ctx.close()
    log1, dims1, spec1, st1 = res[1]
    log0, dims0, spec0, st0 = res[0]
    assert log1 == log0 and dims1 == dims0
    for a, b in zip(spec1, spec0):
        np.testing.assert_allclose(a, b, atol=1e-10, rtol=0)
    assert st1["n_trials_certified"] > 0 and st0["n_trials_certified"] == 0
    assert st1["n_trials"] == st0["n_trials"]

    st = mpo.MPOState(N)
    st.B = [b.copy() for b in B]
    st.lam = [l.copy() for l in lam]
    cfg = mpo.Config(eps=EPS, chi_max=CHI, tau=1e6)
    op = mpo.swap_operator(mpo.SIDE_BOTH)
    want = [b for b in range(0, N - 1, 2) if st.trial(b, op, cfg).count < st.chi(b)]
    got = [rec[3] for rec in log1 if rec[1] == 0 and rec[2] == mpo.SIDE_BOTH and rec[3] % 2 == 0]
    assert got == want
