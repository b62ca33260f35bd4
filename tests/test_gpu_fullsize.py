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
