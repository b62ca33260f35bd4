"""GPU <-> oracle parity at the configurations' own shapes, through the C ABI:

* the precision configuration's bond size chi = 512 (2048 x 2048 bond matrices on the row
  path, 2048 x 1024 on the column path), FP64 and 3xTF32 merges;
* the 28-qubit unswapping configuration's output: the exact peak, its probability and 1000
  samples of the saturated state, against the oracle's search and sampler on the same state;
* the 28-qubit unswapping workload's generator at reduced size (12 qubits) end to end, and the
  HQAP-like workload (RZZ gates, one-qubit layers, swap insertions) at reduced size with the
  paper's cutoff 2e-3 and adaptive sides (App. A.3, A.4), both against the oracle and the
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
    """The 28-qubit unswapping workload's generator at 12 qubits (40 Haar gates per half, a
    random hidden permutation of all 12 qubits, perturbation 0.02, chi_max = 64, eps = 1e-10):
    plans, unswap logs, layouts, bond dimensions, spectra, peak, samples and trace equal the
    oracle's.  At this cap neither finds the planted string although the statevector puts
    most of the weight on it: the random permutation is not undone by adjacent swaps before
    the truncated MPO loses it (the library reproduces the method, including where it fails)."""
    circ = W.hidden_permutation_mirror(12, 40, 0.02, seed=0)
    ref, ctx, c, _ = run_both(circ, eps=1e-10, chi_max=64, tau=3000)
    bits, p = compare_runs(ref, c, circ)
    psi = sv.run_circuit(circ)
    probs = np.abs(psi) ** 2
    s_idx = sum(int(b) << q for q, b in enumerate(circ.planted))
    assert np.argmax(probs) == s_idx and probs[s_idx] > 0.9
    assert not np.array_equal(bits, circ.planted)


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
