"""GPU <-> oracle parity through the C ABI (the CUDA path), element by element on the same
seeded inputs.  Discrete results (bond dimensions, plans, unswap logs, peak bitstrings,
samples) must be identical; floating-point results within the FP64 tolerances stated here:

  TOL_SPEC = 1e-10   bond spectra, absolute (each spectrum has unit 2-norm)
  TOL_PEAK = 1e-12   peak probability, absolute
  TOL_AMP  = 1e-10   amplitudes and two-site tensors, absolute relative to the largest entry

The bound: every update is an FP64 factorisation whose backward error is a few units of
roundoff times the matrix norm (1e-16 .. 1e-14 for the sizes here); the comparisons below
stay four or more orders of magnitude above that, and a dropped term, a wrong index or a
transposed operand moves results by O(1)."""
import numpy as np
import pytest

from oracle import mpo
from oracle import statevector as sv
from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SPEC = 1e-10
TOL_PEAK = 1e-12
TOL_AMP = 1e-10


def random_state(chi, seed):
    """Right-isometric sites (where the shape allows) and geometric spectra."""
    rng = np.random.default_rng(seed)
    n = len(chi) - 1
    B = []
    for j in range(n):
        cl, cr = chi[j], chi[j + 1]
        if cl <= 4 * cr:
            B.append(W.random_right_isometry(rng, cl, cr))
        else:
            z = rng.standard_normal((cl, 4, cr)) + 1j * rng.standard_normal((cl, 4, cr))
            B.append(z / np.linalg.norm(z))
    lam = [W.geometric_spectrum(chi[b + 1], scale=max(2.0, chi[b + 1] / 4)) for b in range(n - 1)]
    return B, lam


def oracle_state(B, lam):
    st = mpo.MPOState(len(B))
    st.B = [b.copy() for b in B]
    st.lam = [l.copy() for l in lam]
    return st


def two_site(Bj, Bj1):
    return np.einsum("lpm,mqr->lpqr", Bj, Bj1)


def ctx_for(**kw):
    return binding.Context(**kw)


def check_update(ctx_kw, chi, bonds, seed, ops=None):
    B, lam = random_state(chi, seed)
    n = len(B)
    rng = np.random.default_rng(seed + 100)
    if ops is None:
        ops = [W.haar_unitary(rng, 16) for _ in bonds]
    ctx = ctx_for(**ctx_kw)
    c = ctx.load_gates(n, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    c.set_state(B, lam)
    got_chi = c.apply_updates(bonds, np.array(ops))
    cfg = mpo.Config(eps=ctx_kw["eps"], chi_max=ctx_kw["chi_max"])
    st = oracle_state(B, lam)
    for k, j in enumerate(bonds):
        t = st.trial(j, ops[k], cfg)
        # guard band: the decision is ambiguous if a singular value sits at the threshold
        thr = cfg.eps * t.s[0]
        near = np.abs(t.s - thr) <= 1e-9 * thr
        assert not near.any(), "seed puts a singular value inside the guard band"
        st.commit(j, t)
        assert got_chi[k] == t.count
        np.testing.assert_allclose(c.spectrum(j), st.lam[j], atol=TOL_SPEC, rtol=0)
        ref = two_site(st.B[j], st.B[j + 1])
        got = two_site(c.site(j), c.site(j + 1))
        assert np.max(np.abs(got - ref)) <= TOL_AMP * max(1.0, np.max(np.abs(ref)))
    # untouched sites are untouched
    touched = {j for b in bonds for j in (b, b + 1)}
    for j in range(n):
        if j not in touched:
            assert np.array_equal(c.site(j), B[j])
    c.close()
    ctx.close()


def test_single_update_ragged_tiles():
    # bond 3: chi_l=37, chi_m=50, chi_r=29 -> a 148 x 116 bond matrix (3 x 2 GEMM tiles, ragged)
    check_update(dict(eps=1e-12, chi_max=256), [1, 4, 13, 37, 50, 29, 11, 4, 1], [3], seed=1)


def test_batched_updates_disjoint_bonds_uneven_sizes():
    check_update(dict(eps=1e-12, chi_max=256), [1, 4, 13, 37, 50, 29, 11, 4, 1], [0, 2, 4, 6], seed=2)


def test_update_with_truncation_active():
    check_update(dict(eps=1e-3, chi_max=20), [1, 4, 13, 20, 20, 19, 11, 4, 1], [1, 3, 5], seed=3)


def test_update_boundary_bonds_and_chi_one():
    check_update(dict(eps=1e-12, chi_max=64), [1, 1, 1, 1, 1], [0, 2], seed=4)
    check_update(dict(eps=1e-12, chi_max=64), [1, 4, 3, 4, 1], [0, 2], seed=5)


def test_permutation_operator_update():
    """A SWAP on the out-legs is a pure permutation of the 16-dim two-site index."""
    ops = [mpo.swap_operator(mpo.SIDE_LEFT), mpo.swap_operator(mpo.SIDE_BOTH)]
    check_update(dict(eps=1e-12, chi_max=256), [1, 4, 16, 30, 16, 4, 1], [1, 3], seed=6, ops=ops)


@pytest.mark.parametrize("seed", [0, 1])
def test_full_size_update_chi256_sampled(seed):
    """The microbenchmark's launch shape: chi_l = chi_m = chi_r = 256 (a 1024 x 1024 bond
    matrix), eps = 1e-10, chi_max = 256; two disjoint updates in one batch."""
    chi = [1, 4, 256, 256, 256, 256, 256, 4, 1]
    check_update(dict(eps=1e-10, chi_max=256), chi, [2, 4], seed=10 + seed)


def run_both(circ, **kw):
    cfg_o = mpo.Config(eps=kw.get("eps", 1e-10), chi_max=kw.get("chi_max", 256), tau=kw.get("tau", 1e6),
                       accept_equal=bool(kw.get("accept_equal", 0)),
                       unswap_parallel=kw.get("unswap_mode", 0) == 0,
                       unswap_enabled=kw.get("unswap_mode", 0) != 2,
                       max_unswap_iter=kw.get("max_unswap_iter", 20))
    ref = mpo.contract(circ, cfg_o)
    ctx = ctx_for(**kw)
    c = ctx.load_circuit(circ)
    stats = c.contract()
    return ref, ctx, c, stats


def compare_runs(ref, c, circ, n_samples=40):
    n = circ.n_qubits
    plan_ref = np.array([[r.side, r.bond, r.kind, r.gate, r.chi] for r in ref.plan], np.int32).reshape(-1, 5)
    assert np.array_equal(c.plan(), plan_ref)
    ul_ref = np.array(ref.unswap_log, np.int32).reshape(-1, 4)
    assert np.array_equal(c.unswap_log(), ul_ref)
    assert list(c.bond_dims()) == ref.state.bond_dims()
    lay_l, lay_r = c.layouts()
    assert list(lay_l) == ref.layout_l.pos and list(lay_r) == ref.layout_r.pos
    for b in range(n - 1):
        np.testing.assert_allclose(c.spectrum(b), ref.state.lam[b], atol=TOL_SPEC, rtol=0)
    out = mpo.project_zero(ref)
    bits_ref, p_ref, _, _ = mpo.extract_peak(out)
    bits, p, norm2 = c.extract_peak()
    assert np.array_equal(bits, bits_ref)
    assert abs(p - p_ref) <= TOL_PEAK
    assert abs(norm2 - out.norm2 * 2 ** n) <= 1e-10
    u = mpo.uniforms(77, n_samples, n)
    samp_ref = mpo.sample(out, u)
    assert np.array_equal(c.sample(n_samples, 77), samp_ref)
    # telemetry (Fig. 3 quantities): the same points as the oracle's trace
    got_tr = [(r["stage"], r["phase"], r["gates"], r["size"], r["max_chi"], r["accepted"]) for r in c.trace()]
    ref_tr = [(t["stage"], 0 if t["phase"] == "absorb" else 1, t["gates"], t["size"], t["max_chi"], t["accepted"])
              for t in ref.trace]
    assert got_tr == ref_tr
    xs = np.vstack([bits_ref[None], np.random.default_rng(0).integers(0, 2, (6, n)).astype(np.uint8)])
    amp_ref = mpo.amplitudes(out, xs)
    assert np.max(np.abs(c.amplitudes(xs) - amp_ref)) <= TOL_AMP
    return bits, p


def test_random_circuit_exact_against_statevector():
    circ = W.random_circuit(6, 18, seed=0)
    ref, ctx, c, _ = run_both(circ, eps=1e-14, chi_max=1024, tau=100)
    compare_runs(ref, c, circ)
    psi = sv.run_circuit(circ)
    xs = np.array([[(x >> q) & 1 for q in range(6)] for x in range(64)], np.uint8)
    assert np.max(np.abs(c.amplitudes(xs) - psi)) <= 1e-12


def test_line12_mirror_collapses_to_bond_dimension_one():
    circ = W.workload_line12(0)
    ref, ctx, c, stats = run_both(circ, eps=1e-12, chi_max=64, tau=1e6)
    assert list(c.bond_dims()) == [1] * 11
    bits, p = compare_runs(ref, c, circ)
    assert np.array_equal(bits, circ.planted) and abs(p - 1.0) <= TOL_PEAK


@pytest.mark.parametrize("n,eps_p,chi_max", [(8, 0.0, 64), (8, 0.02, 64), (9, 0.02, 32)])
def test_hidden_permutation_mirror_end_to_end(n, eps_p, chi_max):
    """Hidden permutation + perturbation; with chi_max = 32 the cap truncates (9 qubits)."""
    circ = W.hidden_permutation_mirror(n, 20, eps_p, seed=1)
    ref, ctx, c, stats = run_both(circ, eps=1e-10, chi_max=chi_max, tau=600)
    assert len(ref.unswap_log) > 0
    bits, p = compare_runs(ref, c, circ)
    assert np.array_equal(bits, circ.planted)


@pytest.mark.parametrize("mode", [1, 0])
def test_permutation_only_both_unswap_variants(mode):
    circ = W.permutation_only(9, seed=3)
    ref, ctx, c, _ = run_both(circ, eps=1e-12, chi_max=256, tau=300, unswap_mode=mode)
    assert list(c.bond_dims()) == [1] * 8
    compare_runs(ref, c, circ)


def test_equal_acceptance_mode():
    circ = W.hidden_permutation_mirror(8, 16, 0.02, seed=4)
    ref, ctx, c, _ = run_both(circ, eps=1e-10, chi_max=256, tau=500, accept_equal=1, max_unswap_iter=3)
    compare_runs(ref, c, circ)


def test_no_two_qubit_gates_only_planted_layer():
    circ = W.permutation_only(5, seed=1)
    circ.pairs = np.zeros((0, 2), np.int32)
    circ.mats = np.zeros((0, 4, 4), complex)
    circ.split_index = 0
    ref, ctx, c, _ = run_both(circ, eps=1e-12, chi_max=16, tau=1e6)
    bits, p = compare_runs(ref, c, circ)
    assert np.array_equal(bits, circ.planted) and abs(p - 1.0) <= TOL_PEAK


def test_errors_are_reported():
    ctx = ctx_for(eps=1e-10, chi_max=16)
    bad = np.eye(4, dtype=complex)[None] * 1.1
    with pytest.raises(binding.PcError) as e:
        ctx.load_gates(3, np.array([[0, 1]]), bad)
    assert e.value.status == -2
    c = ctx.load_gates(6, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    with pytest.raises(binding.PcError) as e:
        c.apply_updates([1, 2], np.stack([np.eye(16)] * 2))
    assert e.value.status == -1


@pytest.mark.parametrize("n,eps_p,seed", [(8, 0.02, 2), (9, 0.03, 3)])
def test_adaptive_side_selection_end_to_end(n, eps_p, seed):
    """App. A.3: each absorption step keeps the side with the smaller size(M); the plans
    (only the kept absorptions), unswap logs, layouts, spectra, peaks and samples must be the
    oracle's."""
    circ = W.hidden_permutation_mirror(n, 20, eps_p, seed=seed)
    ref = mpo.contract(circ, mpo.Config(eps=1e-10, chi_max=64, tau=600, side_adaptive=True))
    assert len(ref.sides) > 0
    ctx = ctx_for(eps=1e-10, chi_max=64, tau=600, side_mode=binding.SIDE_ADAPTIVE)
    c = ctx.load_circuit(circ)
    c.contract()
    compare_runs(ref, c, circ)


def test_checkpoint_file_resume(tmp_path):
    """Contract two outer iterations, write the state to a file, read it into a fresh circuit
    with the same gates and finish there: bond dimensions, layouts, spectra and peak equal an
    uninterrupted run's; a file for another circuit is rejected."""
    circ = W.hidden_permutation_mirror(9, 24, 0.02, seed=6)
    kw = dict(eps=1e-10, chi_max=64, tau=500)
    ctx = ctx_for(**kw)
    full = ctx.load_circuit(circ)
    full.contract()
    a = ctx.load_circuit(circ)
    a.contract_iterations(2)
    path = str(tmp_path / "state.ckpt")
    a.checkpoint_write(path)
    b = ctx.load_circuit(circ)
    b.checkpoint_read(path)
    assert b.cursors() == a.cursors()
    assert list(b.bond_dims()) == list(a.bond_dims())
    b.contract()
    assert list(b.bond_dims()) == list(full.bond_dims())
    assert [x.tolist() for x in b.layouts()] == [x.tolist() for x in full.layouts()]
    for bond in range(circ.n_qubits - 1):
        np.testing.assert_allclose(b.spectrum(bond), full.spectrum(bond), atol=TOL_SPEC, rtol=0)
    bits_b, p_b, _ = b.extract_peak()
    bits_f, p_f, _ = full.extract_peak()
    assert np.array_equal(bits_b, bits_f) and abs(p_b - p_f) <= TOL_PEAK
    other = ctx.load_circuit(W.hidden_permutation_mirror(8, 24, 0.02, seed=6))
    with pytest.raises(binding.PcError) as e:
        other.checkpoint_read(path)
    assert e.value.status == -1


def test_failure_statuses_without_a_fault():
    """Failure detection through status codes, no GPU fault involved: a Jacobi sweep cap of 1
    cannot orthogonalise a random bond matrix (PC_ERR_NOCONVERGE); a circuit with no mirror
    structure keeps size(M) above a tiny tau after unswapping, so the contraction finishes with
    PC_WARN_STALLED (Sec. III.A) exactly where the oracle stalls, with the oracle's result."""
    ctx = ctx_for(eps=1e-10, chi_max=64, jacobi_max_sweeps=1, fp32_precondition=0)
    c = ctx.load_circuit(W.random_circuit(6, 12, seed=1))
    with pytest.raises(binding.PcError) as e:
        c.contract()
    assert e.value.status == -4
    circ = W.random_circuit(6, 20, seed=2)
    ref, ctx2, c2, stats = run_both(circ, eps=1e-10, chi_max=64, tau=50)
    assert ref.stalled
    assert stats["status"] == 1 and stats["stalled"] == 1
    compare_runs(ref, c2, circ)
