"""Pins for the FP64 oracle against things other than itself: brute-force statevector and
full-operator simulation, closed forms, invariants of the mirrored construction, and
exhaustive search on tiny inputs.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mpo
from oracle import statevector as sv
from paper_2604_21908_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EXACT = mpo.Config(eps=1e-14, chi_max=1 << 20, tau=1e12)


def dense_from_mpo(st):
    t = st.B[0]
    for j in range(1, st.n):
        t = np.tensordot(t, st.B[j], axes=([-1], [0]))
    return t.reshape([4] * st.n)


def all_bits(n):
    return np.array([[(x >> q) & 1 for q in range(n)] for x in range(2 ** n)], dtype=np.uint8)


def to_index(bits):
    return sum(int(b) << q for q, b in enumerate(bits))


# --- the generators (inputs) -----------------------------------------------------------

def test_brickwork_mirror_peaks_on_planted():
    c = W.brickwork_mirror(8, 4, seed=3)
    psi = sv.run_circuit(c)
    assert abs(abs(psi[to_index(c.planted)]) ** 2 - 1.0) < 1e-12


@pytest.mark.parametrize("c64", [False, True])
def test_hidden_permutation_mirror_is_identity_up_to_xs(c64):
    c = W.hidden_permutation_mirror(8, 20, 0.0, seed=5, store_complex64=c64)
    assert c.split_index == c.n_gates // 2
    psi = sv.run_circuit(c)
    assert abs(abs(psi[to_index(c.planted)]) ** 2 - 1.0) < 1e-12
    # no SWAP matrix appears verbatim in the gate list
    assert min(np.max(np.abs(m - W.SWAP4)) for m in c.mats) > 1e-3


def test_permutation_transpositions_move_qubits():
    rng = np.random.default_rng(0)
    n = 7
    perm = rng.permutation(n)
    x = rng.integers(0, 2, n)
    psi = np.zeros(2 ** n, complex)
    psi[to_index(x)] = 1
    for a, b in W.permutation_transpositions(perm):
        psi = sv.apply_2q(psi, n, a, b, W.SWAP4)
    y = np.zeros(n, int)
    for q in range(n):
        y[perm[q]] = x[q]
    assert abs(psi[to_index(y)]) == pytest.approx(1.0)


def test_complex64_gates_are_unitary_in_fp64():
    c = W.hidden_permutation_mirror(6, 10, 0.02, seed=1, store_complex64=True)
    for g in c.mats:
        assert np.max(np.abs(g.conj().T @ g - np.eye(4))) < 1e-14


def test_perturbed_mirror_first_order_band():
    """With eps > 0 the peak stays on s and p is near the first-order estimate
    prod_k |tr exp(i eps H_k)/4|^2 (a sanity band, not a pin)."""
    c = W.hidden_permutation_mirror(8, 20, 0.05, seed=2)
    psi = sv.run_circuit(c)
    p = np.abs(psi) ** 2
    assert np.argmax(p) == to_index(c.planted)
    assert 0.8 < p.max() < 1.0


@pytest.mark.parametrize("eps", [0.0, 0.02, 0.05])
def test_perturbation_is_exp_i_eps_h_with_traceless_unit_norm_h(eps):
    """The perturbation of the mirrored half (exp(i eps H), H random Hermitian; the paper does
    not normalise H, the reading here is traceless with unit spectral norm): each gate of V^dagger
    times its original gate of U is exp(i eps H_k), on the relabelled qubits in the same order.
    Its eigenphases divided by eps are H_k's eigenvalues: they sum to 0 and the largest has
    modulus 1.  A Frobenius normalisation, a trace left in, or another exponent convention
    fails this; eps = 0 gives the identity."""
    c = W.hidden_permutation_mirror(6, 10, eps, seed=3, store_complex64=False)
    g, m = c.meta["gates_per_half"], c.meta["n_perm_gates"]
    for k in range(g):
        i = g + m + (g - 1 - k)                      # V^dagger holds U's gates in reverse order
        assert tuple(c.pairs[i]) == (c.permutation[c.pairs[k][0]], c.permutation[c.pairs[k][1]])
        e = c.mats[i] @ c.mats[k]
        assert np.max(np.abs(e.conj().T @ e - np.eye(4))) < 1e-13
        if eps == 0.0:
            assert np.max(np.abs(e - np.eye(4))) < 1e-13
            continue
        lam = np.angle(np.linalg.eigvals(e)) / eps
        assert abs(lam.sum()) < 1e-9
        assert abs(np.max(np.abs(lam)) - 1.0) < 1e-9
        assert np.max(np.abs(lam)) <= 1.0 + 1e-9


# --- single-update math: closed forms --------------------------------------------------

@pytest.mark.parametrize("name", ["SWAP", "CNOT", "product"])
def test_one_gate_operator_schmidt_closed_form(name):
    with open(os.path.join(GOLDEN, "operator_schmidt.json")) as f:
        gold = json.load(f)
    rng = np.random.default_rng(1)
    if name == "SWAP":
        g = W.SWAP4
    elif name == "CNOT":
        g = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)
    else:
        g = np.kron(W.haar_unitary(rng, 2), W.haar_unitary(rng, 2))
    for side in (mpo.SIDE_LEFT, mpo.SIDE_RIGHT):
        st = mpo.MPOState(2)
        u16 = mpo.two_site_operator(g, None) if side == mpo.SIDE_LEFT else mpo.two_site_operator(None, g)
        st.apply(0, u16, mpo.Config(eps=1e-12))
        np.testing.assert_allclose(st.lam[0], gold[name], atol=1e-14)


def test_two_site_operator_is_g_kron_h_transpose():
    """On vec(M) with per-site index p = 2o + i, M <- g M h is a unitary 16x16 operator;
    check it against the definition written with explicit loops."""
    rng = np.random.default_rng(2)
    g, h = W.haar_su4(rng), W.haar_su4(rng)
    u = mpo.two_site_operator(g, h)
    assert np.max(np.abs(u.conj().T @ u - np.eye(16))) < 1e-13
    m = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))   # M[(o1 o2), (i1 i2)]
    m_new = g @ m @ h
    vec = np.zeros(16, complex)
    for o1, i1, o2, i2 in np.ndindex(2, 2, 2, 2):
        vec[4 * (2 * o1 + i1) + (2 * o2 + i2)] = m[2 * o1 + o2, 2 * i1 + i2]
    out = u @ vec
    for o1, i1, o2, i2 in np.ndindex(2, 2, 2, 2):
        assert abs(out[4 * (2 * o1 + i1) + (2 * o2 + i2)] - m_new[2 * o1 + o2, 2 * i1 + i2]) < 1e-13


def test_truncation_count_rule():
    s = np.array([1.0, 0.5, 1e-10, 2e-10, 0.0])
    s = np.sort(s)[::-1]
    assert mpo.truncation_count(s, 1e-10, 100) == 3      # strict '>' at the cutoff
    assert mpo.truncation_count(s, 1e-10, 2) == 2        # chi_max cap
    assert mpo.truncation_count(np.zeros(3), 1e-10, 5) == 1


# --- the contraction against brute force ---------------------------------------------

@pytest.mark.parametrize("seed,line", [(0, False), (1, True), (2, False)])
def test_dense_mpo_equals_circuit_operator(seed, line):
    c = W.random_circuit(6, 14, seed=seed, line=line)
    r = mpo.contract(c, EXACT)
    op = sv.full_operator(c)
    t_ref = sv.operator_to_sites(op, 6, r.layout_l.pos, r.layout_r.pos) / 2 ** 3
    assert np.max(np.abs(dense_from_mpo(r.state) - t_ref)) < 1e-12
    for cut in range(5):
        s_ref = sv.operator_schmidt_values(t_ref, cut)
        k = len(r.state.lam[cut])
        assert np.max(np.abs(s_ref[:k] - r.state.lam[cut])) < 1e-12
        assert np.all(s_ref[k:] < 1e-13)
        assert abs(np.sum(r.state.lam[cut] ** 2) - 1.0) < 1e-13


def test_unswap_keeps_the_operator():
    """Unswapping only moves permutation content into the layouts (Eq. 1): with the cutoff
    inactive the MPO with its layouts still equals the circuit's operator."""
    c = W.random_circuit(6, 16, seed=7)
    cfg = mpo.Config(eps=1e-14, chi_max=1 << 20, tau=40)
    r = mpo.contract(c, cfg)
    assert len(r.unswap_log) > 0
    op = sv.full_operator(c)
    t_ref = sv.operator_to_sites(op, 6, r.layout_l.pos, r.layout_r.pos) / 2 ** 3
    assert np.max(np.abs(dense_from_mpo(r.state) - t_ref)) < 1e-12


@pytest.mark.parametrize("n,n_gates,tau,seed", [(6, 18, 100, 0), (9, 7, 1e12, 1)])
def test_amplitudes_and_peak_match_statevector(n, n_gates, tau, seed):
    c = W.random_circuit(n, n_gates, seed=seed)
    r = mpo.contract(c, mpo.Config(eps=1e-14, chi_max=1 << 20, tau=tau))
    m = mpo.project_zero(r)
    psi = sv.run_circuit(c)
    amp = mpo.amplitudes(m, all_bits(n))
    assert np.max(np.abs(amp - psi)) < 1e-12
    assert abs(m.norm2 * 2 ** n - 1.0) < 1e-12
    bits, p, p_raw, _ = mpo.extract_peak(m)
    assert to_index(bits) == int(np.argmax(np.abs(psi) ** 2))
    assert abs(p - np.max(np.abs(psi) ** 2)) < 1e-12


def test_sampling_is_inverse_cdf_of_statevector():
    n = 6
    c = W.random_circuit(n, 10, seed=4)
    r = mpo.contract(c, mpo.Config(eps=1e-14, chi_max=1 << 20, tau=100))
    m = mpo.project_zero(r)
    probs = np.abs(sv.run_circuit(c)) ** 2
    site_of = r.layout_l.pos
    xs = all_bits(n)
    ys = np.array([[x[r.layout_l.site[j]] for j in range(n)] for x in xs])   # site bits
    u = mpo.uniforms(11, 40, n)
    got = mpo.sample(m, u)
    for s in range(u.shape[0]):
        mask = np.ones(2 ** n, bool)
        y = []
        for j in range(n):
            p0 = probs[mask & (ys[:, j] == 0)].sum() / probs[mask].sum()
            b = 1 if u[s, j] >= p0 else 0
            y.append(b)
            mask &= ys[:, j] == b
        x = [y[site_of[q]] for q in range(n)]
        assert list(got[s]) == x


def test_mirror_invariant_brickwork12():
    """Unperturbed U^dagger U: every bond returns to dimension 1, M = (x)_q X^{s_q},
    the peak is s with probability 1 (the 12-qubit line workload)."""
    c = W.workload_line12(0)
    r = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=64, tau=1e6))
    assert r.state.bond_dims() == [1] * 11
    m = mpo.project_zero(r)
    bits, p, _, _ = mpo.extract_peak(m)
    assert (bits == c.planted).all()
    assert abs(p - 1.0) < 1e-12
    psi = sv.run_circuit(c)
    assert abs(abs(psi[to_index(c.planted)]) ** 2 - 1.0) < 1e-12


def test_trace_of_the_mirror_cancels_layer_pair_by_layer_pair():
    """Fig. 3 telemetry on the unperturbed brickwork mirror, one layer pair per outer iteration
    (tau = 1): absorbing the innermost layer of C_L (an adjoint layer of U) and of C_R (the same
    layer of U) multiplies M by U_t^dagger ... U_t, so M returns to the identity after every
    stage: each absorb record has every bond at dimension 1 (size(M) = 4n) and the two-qubit
    gates absorbed grow by twice the brickwork layer size, counted here from the gate list
    (layers of U alternate 6 and 5 gates on 12 qubits; the innermost is U's last)."""
    n, layers = 12, 8
    c = W.brickwork_mirror(n, layers, seed=4)
    sizes = [len(range(t % 2, n - 1, 2)) for t in range(layers)]         # U's layers in time order
    expect = list(2 * np.cumsum(sizes[::-1]))
    r = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=64, tau=1))
    absorb = [rec for rec in r.trace if rec["phase"] == "absorb"]
    assert len(absorb) >= layers
    assert [rec["gates"] for rec in absorb[:layers]] == expect
    for rec in absorb:
        assert rec["size"] == 4 * n and rec["max_chi"] == 1
    assert all(rec["accepted"] == 0 for rec in r.trace)
    assert r.trace[-1]["gates"] == 2 * sum(sizes)


@pytest.mark.parametrize("parallel", [True, False])
def test_permutation_only_unswaps_to_product(parallel):
    """C = X^s P_pi as a SWAP network: unswapping extracts the whole permutation, every
    bond ends at dimension 1 and the peak is s with probability 1."""
    c = W.permutation_only(9, seed=3)
    cfg = mpo.Config(eps=1e-12, chi_max=256, tau=300, unswap_parallel=parallel)
    r = mpo.contract(c, cfg)
    assert r.state.bond_dims() == [1] * 8
    m = mpo.project_zero(r)
    bits, p, _, _ = mpo.extract_peak(m)
    assert (bits == c.planted).all() and abs(p - 1.0) < 1e-12


def test_hidden_permutation_unswap_recovers_peak():
    c = W.hidden_permutation_mirror(8, 20, 0.0, seed=1)
    r = mpo.contract(c, mpo.Config(eps=1e-10, chi_max=256, tau=600))
    assert len(r.unswap_log) > 0
    assert r.state.bond_dims() == [1] * 7
    m = mpo.project_zero(r)
    bits, p, _, _ = mpo.extract_peak(m)
    assert (bits == c.planted).all() and abs(p - 1.0) < 1e-12


def test_strict_unswap_decreases_total_bond_dimension():
    c = W.random_circuit(6, 14, seed=9)
    cfg = mpo.Config(eps=1e-12, chi_max=1 << 20, tau=1e12)
    ctr = mpo.Contraction(c, cfg)
    while ctr.layers_remain():
        ctr._absorb_left_layer()
        ctr._absorb_right_layer()
    orig_commit = ctr.state.commit
    seen = []

    def commit(j, t):
        before = sum(ctr.state.bond_dims())
        orig_commit(j, t)
        seen.append(sum(ctr.state.bond_dims()) < before)
    ctr.state.commit = commit
    ctr.unswap_parallel()
    assert all(seen)


def test_unswap_trial_counts_match_brute_force():
    """Each trial's count equals the operator-Schmidt rank of the swapped operator, from
    the full 4^n tensor (exhaustive over bonds and sides, n = 5)."""
    n = 5
    c = W.random_circuit(n, 8, seed=12)
    cfg = mpo.Config(eps=1e-9, chi_max=1 << 20, tau=1e12)
    r = mpo.contract(c, cfg)
    t = dense_from_mpo(r.state)
    for i in range(n - 1):
        for side in (mpo.SIDE_LEFT, mpo.SIDE_RIGHT, mpo.SIDE_BOTH):
            tr = r.state.trial(i, mpo.swap_operator(side), cfg)
            u = mpo.swap_operator(side).reshape(4, 4, 4, 4)
            t2 = np.moveaxis(np.tensordot(u, t, axes=([2, 3], [i, i + 1])), [0, 1], [i, i + 1])
            s = sv.operator_schmidt_values(t2, i)
            assert tr.count == mpo.truncation_count(s, cfg.eps, cfg.chi_max)


def test_truncated_update_is_idempotent():
    """Right after a truncating update of bond j, B[j+1] = V^dagger exactly, so merging
    again gives the singular values lam[j] and the same count (truncation is idempotent)."""
    c = W.random_circuit(6, 12, seed=5)
    cfg = mpo.Config(eps=1e-3, chi_max=8, tau=1e12)
    r = mpo.contract(c, cfg)
    st = r.state
    rng = np.random.default_rng(3)
    for j in range(5):
        st.apply(j, mpo.two_site_operator(W.haar_su4(rng), None), cfg)
        lam = st.lam[j].copy()
        assert abs(np.sum(lam ** 2) - 1.0) < 1e-13
        k = st.apply(j, np.eye(16, dtype=complex), cfg)
        assert k == len(lam)
        assert np.max(np.abs(st.lam[j] - lam)) < 1e-12


def test_splitmix64_uniforms():
    u = mpo.uniforms(2026, 2000, 5)
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u.ravel(), bins=10, range=(0, 1))
    chi2 = np.sum((hist - 1000) ** 2 / 1000)
    assert chi2 < 30.0                       # 9 dof, p ~ 4e-4
    assert len(set(u.ravel().tolist())) == u.size


def test_layers_are_disjoint_and_ordered():
    c = W.random_circuit(9, 40, seed=1)
    layers = mpo.layers_from(list(range(c.n_gates)), c.pairs)
    seen_q = {}
    for li, layer in enumerate(layers):
        qs = [q for g in layer for q in c.pairs[g]]
        assert len(qs) == len(set(qs))
        assert layer == sorted(layer)
        for g in layer:
            for q in c.pairs[g]:
                assert seen_q.get(int(q), -1) < li
        for g in layer:
            for q in c.pairs[g]:
                seen_q[int(q)] = li
    assert sorted(g for layer in layers for g in layer) == list(range(c.n_gates))


# --- App. A.3 adaptive side selection ---------------------------------------------------

@pytest.mark.parametrize("seed,tau", [(3, 1e12), (4, 40)])
def test_adaptive_order_keeps_the_circuit_operator(seed, tau):
    """Left and right absorptions act on different legs and commute, so any absorption order
    (here the adaptive one, with and without unswapping) ends at the circuit's operator."""
    c = W.random_circuit(6, 16, seed=seed)
    cfg = mpo.Config(eps=1e-14, chi_max=1 << 20, tau=tau, side_adaptive=True)
    r = mpo.contract(c, cfg)
    assert len(r.sides) > 0
    op = sv.full_operator(c)
    t_ref = sv.operator_to_sites(op, 6, r.layout_l.pos, r.layout_r.pos) / 2 ** 3
    assert np.max(np.abs(dense_from_mpo(r.state) - t_ref)) < 1e-12
    psi = sv.run_circuit(c)
    bits, p, _, _ = mpo.extract_peak(mpo.project_zero(r))
    assert to_index(bits) == int(np.argmax(np.abs(psi) ** 2))
    assert abs(p - np.max(np.abs(psi) ** 2)) < 1e-12


def test_adaptive_mirror_collapses_and_peaks_on_planted():
    c = W.hidden_permutation_mirror(8, 16, 0.0, seed=2)
    r = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=64, tau=300, side_adaptive=True))
    assert r.state.bond_dims() == [1] * 7
    bits, p, _, _ = mpo.extract_peak(mpo.project_zero(r))
    assert np.array_equal(bits, c.planted) and abs(p - 1.0) < 1e-12


def test_adaptive_step_keeps_the_smaller_size():
    """Each adaptive step leaves size(M) at the smaller of the two one-sided absorptions
    (ties to the left), and the sides differ from plain alternation on this circuit."""
    c = W.hidden_permutation_mirror(7, 14, 0.03, seed=5)
    cfg = mpo.Config(eps=1e-10, chi_max=64, tau=1e12, side_adaptive=True, unswap_enabled=False)
    ctr = mpo.Contraction(c, cfg)
    sides = []
    while ctr.layers_remain():
        can_l = ctr.left_cursor < len(ctr.left_layers) or not ctr.oneq_done
        can_r = ctr.right_cursor < len(ctr.right_layers)
        sizes = {}
        if can_l and can_r:
            for side in (mpo.SIDE_LEFT, mpo.SIDE_RIGHT):
                probe = mpo.Contraction(c, cfg)
                probe._load(ctr._save())
                (probe._absorb_left_layer if side == mpo.SIDE_LEFT else probe._absorb_right_layer)()
                sizes[side] = probe.state.size()
        side = ctr._absorb_step_adaptive()
        sides.append(side)
        if sizes:
            assert ctr.state.size() == min(sizes.values())
            assert side == (mpo.SIDE_LEFT if sizes[mpo.SIDE_LEFT] <= sizes[mpo.SIDE_RIGHT] else mpo.SIDE_RIGHT)
    alternate = [mpo.SIDE_LEFT, mpo.SIDE_RIGHT] * len(sides)
    assert sides != alternate[: len(sides)]


def test_adaptive_plan_holds_the_kept_absorptions():
    """The plan of an adaptive run, cut at the steps, replays to the same MPO: each step's
    records are the updates of the side it kept (left = out-legs, right = in-legs)."""
    c = W.hidden_permutation_mirror(7, 14, 0.03, seed=5)
    cfg = mpo.Config(eps=1e-10, chi_max=64, tau=1e12, side_adaptive=True, unswap_enabled=False)
    r = mpo.contract(c, cfg)
    # replay: apply the recorded operators in order on a fresh identity MPO
    st = mpo.MPOState(c.n_qubits)
    lay = {mpo.SIDE_LEFT: mpo.Layout(c.n_qubits), mpo.SIDE_RIGHT: mpo.Layout(c.n_qubits)}
    for rec in r.plan:
        if rec.kind == 0:
            st.apply(rec.bond, mpo.swap_operator(rec.side), cfg)
            lay[rec.side].swap_sites(rec.bond)
        else:
            a, b = int(c.pairs[rec.gate, 0]), int(c.pairs[rec.gate, 1])
            gate = c.mats[rec.gate]
            if lay[rec.side].pos[a] > lay[rec.side].pos[b]:
                gate = mpo.SWAP4 @ gate @ mpo.SWAP4
            u16 = mpo.two_site_operator(gate, None) if rec.side == mpo.SIDE_LEFT else mpo.two_site_operator(None, gate)
            st.apply(rec.bond, u16, cfg)
    for q, g2 in zip(c.oneq_qubits, c.oneq_mats):
        st.apply_one_site(lay[mpo.SIDE_LEFT].pos[int(q)], g2, mpo.SIDE_LEFT)
    assert st.bond_dims() == r.state.bond_dims()
    assert np.max(np.abs(dense_from_mpo(st) - dense_from_mpo(r.state))) < 1e-12


def test_best_first_peak_equals_exhaustive_argmax_n12():
    """Best-first search over prefix marginals returns the exhaustive argmax of |<x|C|0>|^2
    (here a strongly perturbed 12-qubit mirror whose peak is far below 1)."""
    c = W.hidden_permutation_mirror(12, 6, 0.5, seed=8)
    r = mpo.contract(c, mpo.Config(eps=1e-13, chi_max=4096, tau=1e12))
    m = mpo.project_zero(r)
    psi = sv.run_circuit(c)
    probs = np.abs(psi) ** 2
    bits, p, _, _ = mpo.extract_peak(m)
    assert to_index(bits) == int(np.argmax(probs))
    assert abs(p - probs.max()) < 1e-12
    assert probs.max() < 0.9


def test_input_side_permutation_changes_no_amplitude():
    """P_R acts on |0...0> first and P|0...0> = |0...0>: a SWAP network placed before a circuit
    (the outermost part of C_R) leaves every amplitude of C|0> unchanged (Eq. 1)."""
    base = W.random_circuit(6, 12, seed=9)
    rng = np.random.default_rng(3)
    swaps = [tuple(int(q) for q in rng.choice(6, 2, replace=False)) for _ in range(5)]
    pairs = np.vstack([np.array(swaps, np.int32), base.pairs])
    mats = np.concatenate([np.stack([mpo.SWAP4] * len(swaps)), base.mats])
    pre = W.Circuit(6, pairs, mats, base.split_index + len(swaps), base.oneq_qubits, base.oneq_mats)
    amps = []
    for c in (base, pre):
        r = mpo.contract(c, mpo.Config(eps=1e-14, chi_max=1 << 20, tau=30))
        amps.append(mpo.amplitudes(mpo.project_zero(r), all_bits(6)))
    assert np.max(np.abs(amps[0] - amps[1])) < 1e-12
    assert np.max(np.abs(amps[0] - sv.run_circuit(base))) < 1e-12


@pytest.mark.parametrize("parallel", [True, False])
def test_unswapped_layouts_reproduce_the_permutation(parallel):
    """Eq. 1 on a permutation-only circuit C = X^s P_pi: once every bond is at dimension 1 the
    whole permutation sits in the layouts.  A basis state with a single 1 on input qubit q
    enters at site layout_R[q] and leaves from the qubit the left layout puts at that site; the
    statevector of C (without the X^s layer) says where that 1 goes."""
    c = W.permutation_only(8, seed=5, planted=False)
    r = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=256, tau=100, unswap_parallel=parallel))
    assert r.state.bond_dims() == [1] * 7
    site_to_out = {s: q for q, s in enumerate(r.layout_l.pos)}
    for q in range(8):
        psi0 = np.zeros(2 ** 8, np.complex128)
        psi0[1 << q] = 1.0
        psi = sv.run_circuit(c, psi0)
        out = int(np.argmax(np.abs(psi)))
        assert abs(abs(psi[out]) - 1.0) < 1e-12
        assert out == 1 << site_to_out[r.layout_r.pos[q]]


# --- the HQAP-like workload (RZZ gates, one-qubit layers, swap insertions) ----------------

def test_swap_as_native_gates_is_a_swap():
    rng = np.random.default_rng(11)
    g = W.swap_as_native_gates(rng)
    assert len(g) == 3
    assert np.max(np.abs(g[2] @ g[1] @ g[0] - W.SWAP4)) < 1e-14
    for x in g:
        assert np.max(np.abs(x.conj().T @ x - np.eye(4))) < 1e-14
        assert np.max(np.abs(x - W.SWAP4)) > 1e-3


def test_rzz_is_exp_of_zz():
    theta = 0.7
    zz = np.diag([1.0, -1.0, -1.0, 1.0])
    assert np.max(np.abs(W.rzz(theta) - np.diag(np.exp(-0.5j * theta * np.diag(zz))))) < 1e-15


def test_hqap_like_mirror_peaks_on_planted():
    """Without angle noise C|0> = |s>; with it the planted string keeps most of the weight,
    near the first-order estimate exp(-g sigma^2 / 4) (a sanity band)."""
    c = W.hqap_like_mirror(10, 40, 3, 0.0, seed=2)
    assert c.split_index == c.n_gates // 2 and c.n_gates == 2 * 40 + 9
    psi = sv.run_circuit(c)
    assert abs(abs(psi[to_index(c.planted)]) ** 2 - 1.0) < 1e-12
    c = W.hqap_like_mirror(10, 40, 3, 0.1, seed=2)
    p = np.abs(sv.run_circuit(c)) ** 2
    assert np.argmax(p) == to_index(c.planted)
    assert 0.75 < p.max() < 1.0


def test_oracle_contracts_hqap_like_exactly():
    """The oracle on an HQAP-like circuit with the cutoff inactive reproduces every amplitude of
    the statevector (n = 8)."""
    c = W.hqap_like_mirror(8, 24, 2, 0.1, seed=4)
    r = mpo.contract(c, mpo.Config(eps=1e-14, chi_max=1 << 20, tau=200))
    amps = mpo.amplitudes(mpo.project_zero(r), all_bits(8))
    assert np.max(np.abs(amps - sv.run_circuit(c))) < 1e-11


# --- recanonicalisation (Algorithm 1: compress M to canonical form) -----------------------

def test_recanonicalise_restores_vidal_form_of_a_truncated_state():
    """After truncating updates the stored lam drift from the Schmidt values of the operator
    the sites hold; recanonicalisation (cutoff inactive) keeps that operator (up to the norm)
    and makes every B right-canonical with lam = its operator-Schmidt values across each cut
    (brute force on the dense 4^n tensor)."""
    c = W.random_circuit(6, 16, seed=3)
    r = mpo.contract(c, mpo.Config(eps=1e-3, chi_max=6, tau=1e12, recanonicalise=False))
    st = r.state
    t0 = dense_from_mpo(st)
    t0 = t0 / np.linalg.norm(t0)
    drift = max(np.max(np.abs(sv.operator_schmidt_values(t0, j)[:len(st.lam[j])] - st.lam[j])) for j in range(5))
    assert drift > 1e-3                     # the truncated Hastings form has drifted
    st.recanonicalise(mpo.Config(eps=1e-14, chi_max=1 << 20))
    t1 = dense_from_mpo(st)
    assert np.max(np.abs(t1 / np.linalg.norm(t1) - t0)) < 1e-12
    for j in range(6):
        m = st.B[j].reshape(st.B[j].shape[0], -1)
        if j > 0:
            assert np.max(np.abs(m @ m.conj().T - np.eye(m.shape[0]))) < 1e-12
    for j in range(5):
        s_ref = sv.operator_schmidt_values(t0, j)
        k = len(st.lam[j])
        assert np.max(np.abs(st.lam[j] - s_ref[:k])) < 1e-12
        assert np.all(s_ref[k:] < 1e-12)


def test_recanonicalise_is_the_identity_on_an_exact_vidal_state():
    c = W.random_circuit(6, 14, seed=0)
    r = mpo.contract(c, mpo.Config(eps=1e-14, chi_max=1 << 20, tau=1e12))
    lam = [l.copy() for l in r.state.lam]
    t0 = dense_from_mpo(r.state)
    r.state.recanonicalise(mpo.Config(eps=1e-14, chi_max=1 << 20))
    assert np.max(np.abs(dense_from_mpo(r.state) - t0)) < 1e-13
    for a, b in zip(lam, r.state.lam):
        assert np.max(np.abs(a - b)) < 1e-13
