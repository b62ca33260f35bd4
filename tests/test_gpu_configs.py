"""GPU <-> oracle parity at the configurations' own shapes, through the C ABI:

* the precision configuration's bond size chi = 512 (2048 x 2048 bond matrices on the row
  path, 2048 x 1024 on the column path), FP64 and 3xTF32 merges;
* the 28-qubit unswapping configuration's output: the exact peak, its probability and 1000
  samples of the saturated state, against the oracle's search and sampler on the same state;
* the 28-qubit unswapping workload's generator at reduced size end to end (10 qubits: solved;
  12 qubits: where the method fails and only the discrete results are determined), and the
  HQAP-like workload (RZZ gates, one-qubit layers, swap insertions) at reduced size with the
  paper's cutoff 2e-3 and adaptive sides (App. A.3, A.4), against the oracle and the
  statevector.
Tolerances as in test_gpu_parity (FP64) and test_gpu_mixed (mixed precision)."""
import numpy as np
import pytest

from oracle import mpo
from oracle import statevector as sv
from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

from test_gpu_parity import TOL_AMP, TOL_PEAK, check_update, compare_runs, run_both
from test_gpu_mixed import check_mixed_update

pytestmark = pytest.mark.gpu

CHI512 = [1, 4, 16, 64, 256, 512, 512, 512, 256, 64, 16, 4, 1]


def test_chi512_row_path_fp64():
    """Bond 5: chi_l = chi_m = chi_r = 512, a 2048 x 2048 bond matrix (FP32 sweeps on rows
    longer than 1024 use the row-pair kernel), cap active at 512."""
    check_update(dict(eps=1e-10, chi_max=512), CHI512, [5], seed=21)


def test_chi512_column_path_fp64():
    """Bond 6: chi_l = 512, chi_r = 256, a 2048 x 1024 bond matrix factorised through its
    1024 columns (rotations accumulated into the right singular vectors)."""
    check_update(dict(eps=1e-10, chi_max=512), CHI512, [6], seed=22)


def test_chi512_mixed_merge():
    """The same 2048 x 2048 update with the 3xTF32 tensor-core merge (K = 512: 32 K-stages)."""
    check_mixed_update(CHI512, [5], seed=23, chi_max=512)


def test_unswap28_saturated_peak_and_samples():
    """The 28-qubit state of the unswapping configuration's saturated regime: the library's
    exact peak search, p_peak and 1000 samples (fixed uniforms) equal the oracle's."""
    n = 28
    B, lam = W.peaked_saturated_state(n, 256, 0)
    ctx = binding.Context(eps=1e-10, chi_max=256, tau=1e6)
    c = ctx.load_gates(n, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    c.set_state(B, lam)
    st = mpo.MPOState(n)
    st.B = [b.copy() for b in B]
    st.lam = [l.copy() for l in lam]
    out = mpo.project_zero(mpo.Result(st, mpo.Layout(n), mpo.Layout(n)))
    bits_ref, p_ref, _, _ = mpo.extract_peak(out)
    bits, p, norm2 = c.extract_peak()
    assert np.array_equal(bits, bits_ref)
    assert abs(p - p_ref) <= TOL_PEAK
    assert abs(norm2 - out.norm2 * 2 ** n) <= 1e-10 * out.norm2 * 2 ** n
    u = mpo.uniforms(77, 1000, n)
    assert np.array_equal(c.sample(1000, 77), mpo.sample(out, u))
    xs = np.vstack([bits_ref[None], np.random.default_rng(5).integers(0, 2, (7, n)).astype(np.uint8)])
    amp_ref = mpo.amplitudes(out, xs)
    assert np.max(np.abs(c.amplitudes(xs) - amp_ref)) <= TOL_AMP * np.max(np.abs(amp_ref))
    c.close()
    ctx.close()


def test_unswap28_generator_reduced_end_to_end():
    """The 28-qubit unswapping workload's generator at 10 qubits (30 Haar gates per half, a random
    hidden permutation of all 10 qubits, perturbation 0.02, chi_max = 64, eps = 1e-10, tau = 3000):
    plans, unswap logs, layouts, bond dimensions, spectra, peak, samples and trace equal the
    oracle's, and the peak is the planted string (the statevector's argmax)."""
    circ = W.hidden_permutation_mirror(10, 30, 0.02, seed=0)
    ref, ctx, c, _ = run_both(circ, eps=1e-10, chi_max=64, tau=3000)
    bits, p = compare_runs(ref, c, circ)
    assert np.array_equal(bits, circ.planted)
    probs = np.abs(sv.run_circuit(circ)) ** 2
    assert int(np.argmax(probs)) == sum(int(b) << q for q, b in enumerate(circ.planted))


def test_unswap28_generator_where_the_method_fails():
    """At 12 qubits (40 gates per half, chi_max = 64) the random hidden permutation is not undone
    by adjacent swaps before the truncated MPO loses it: the statevector puts most of the weight
    on the planted string, the method keeps a few per cent of it at best.  Every cut there is
    truncated at the cap with near-degenerate singular values, so only the discrete results are
    determined: the oracle itself, with LAPACK's divide-and-conquer SVD in place of gesvd, keeps
    the same plan but moves the final spectra by 0.1 and changes the peak.  Compared: plans
    (with the bond dimension after every update), unswap logs, layouts and bond dimensions; the
    library's spectra are checked to be normalised and sorted, its peak probability small."""
    circ = W.hidden_permutation_mirror(12, 40, 0.02, seed=0)
    ref, ctx, c, _ = run_both(circ, eps=1e-10, chi_max=64, tau=3000)
    plan_ref = np.array([[r.side, r.bond, r.kind, r.gate, r.chi] for r in ref.plan], np.int32).reshape(-1, 5)
    assert np.array_equal(c.plan(), plan_ref)
    assert np.array_equal(c.unswap_log(), np.array(ref.unswap_log, np.int32).reshape(-1, 4))
    lay_l, lay_r = c.layouts()
    assert list(lay_l) == ref.layout_l.pos and list(lay_r) == ref.layout_r.pos
    assert list(c.bond_dims()) == ref.state.bond_dims()
    for b in range(circ.n_qubits - 1):
        s = c.spectrum(b)
        assert abs(np.sum(s ** 2) - 1.0) < 1e-12 and np.all(np.diff(s) <= 1e-15)
    bits, p, norm2 = c.extract_peak()
    assert 0.0 < p < 0.5
    probs = np.abs(sv.run_circuit(circ)) ** 2
    s_idx = sum(int(b) << q for q, b in enumerate(circ.planted))
    assert np.argmax(probs) == s_idx and probs[s_idx] > 0.9


def test_hqap_like_reduced_end_to_end():
    """The HQAP-like workload at 12 qubits (60 RZZ gates per half, three swap insertions, angle
    noise 0.1) with the paper's cutoff 2e-3, strict acceptance and adaptive sides: everything
    equals the oracle's, and the peak is the planted string (the statevector's argmax)."""
    circ = W.hqap_like_mirror(12, 60, 3, 0.1, seed=0)
    ref = mpo.contract(circ, mpo.Config(eps=2e-3, chi_max=64, tau=3000, side_adaptive=True))
    ctx = binding.Context(eps=2e-3, chi_max=64, tau=3000, side_mode=binding.SIDE_ADAPTIVE)
    c = ctx.load_circuit(circ)
    c.contract()
    bits, p = compare_runs(ref, c, circ)
    assert np.array_equal(bits, circ.planted)
    psi = sv.run_circuit(circ)
    assert int(np.argmax(np.abs(psi) ** 2)) == sum(int(b) << q for q, b in enumerate(circ.planted))
