"""Pins for the oracle's discrete decisions, against computations that share nothing with
it: the sequential (Algorithm 1) and parallel (App. A.1) unswap rules replayed on the dense 4^n
operator built from the statevector simulator, the stall flag on circuits whose size(M) is fixed by construction,
and the counter-based SplitMix64 stream against its published outputs.  CPU only."""
import math

import numpy as np
import pytest

from oracle import mpo
from oracle import statevector as sv
from paper_2604_21908_gb300 import workloads as W


# --- SplitMix64 (Steele, Lea, Flood 2014) ------------------------------------------------

def test_splitmix64_published_outputs():
    """The generator stepped from seed 1234567 has the published first five outputs, and
    floor(5 x / 2^64) over 100,000 outputs from seed 987654321 has the published bucket
    counts.  splitmix64(seed, k) is the (k+1)-th output of the generator started at seed."""
    first = [mpo.splitmix64(1234567, k) for k in range(5)]
    assert first == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                     4593380528125082431, 16408922859458223821]
    counts = [0] * 5
    for k in range(100000):
        counts[(mpo.splitmix64(987654321, k) * 5) >> 64] += 1
    assert counts == [20027, 19892, 20073, 19978, 20030]


def test_uniforms_are_top_53_bits():
    """u[s][j] = (output >> 11) * 2^-53: exactly representable, in [0, 1)."""
    u = mpo.uniforms(1234567, 1, 5)
    for k in range(5):
        assert u[0, k] == (mpo.splitmix64(1234567, k) >> 11) / 2.0 ** 53


# --- sequential unswapping (Algorithm 1) replayed on the dense operator ------------------

def _count(s, eps, chi_max):
    # the cutoff rule (Sec. II.B.1, App. A.4): s_k > eps * s_0, at least 1, at most chi_max
    if s[0] <= 0:
        return 1
    return max(1, min(int(np.sum(s > eps * s[0])), chi_max))


def _swap_legs(t, n, bond, side):
    """A SWAP taken into M on sites (bond, bond+1): from the left it exchanges the two
    output legs, from the right the two input legs, from both sides both pairs."""
    t = t.reshape([2] * (2 * n))                  # axes (o_0, i_0, o_1, i_1, ...)
    perm = list(range(2 * n))
    if side in (mpo.SIDE_LEFT, mpo.SIDE_BOTH):
        perm[2 * bond], perm[2 * bond + 2] = perm[2 * bond + 2], perm[2 * bond]
    if side in (mpo.SIDE_RIGHT, mpo.SIDE_BOTH):
        perm[2 * bond + 1], perm[2 * bond + 3] = perm[2 * bond + 3], perm[2 * bond + 1]
    return np.transpose(t, perm).reshape([4] * n)


def _replay_sequential(t, n, eps, chi_max, equal, cap, pos_l=None, pos_r=None):
    """Algorithm 1's unswapping on the dense site tensor: the available bond of largest
    operator-Schmidt rank (smallest index on ties), its three swapped variants ranked by
    rank with ties left < right < both, accepted when the rank drops (or does not grow, in
    equal mode); an accepted bond leaves the available set and its neighbours rejoin it, a
    rejected one just leaves it."""
    avail = set(range(n - 1))
    log, steps = [], 0
    pos = {mpo.SIDE_LEFT: list(pos_l if pos_l is not None else range(n)),
           mpo.SIDE_RIGHT: list(pos_r if pos_r is not None else range(n))}
    while avail and steps < cap:
        steps += 1
        ranks = [_count(sv.operator_schmidt_values(t, b), eps, chi_max) for b in range(n - 1)]
        i = min(avail, key=lambda b: (-ranks[b], b))
        cands = []
        for side in (mpo.SIDE_LEFT, mpo.SIDE_RIGHT, mpo.SIDE_BOTH):
            t2 = _swap_legs(t, n, i, side)
            cands.append((_count(sv.operator_schmidt_values(t2, i), eps, chi_max), side, t2))
        best = min(cands, key=lambda c: (c[0], c[1]))
        ok = best[0] <= ranks[i] if equal else best[0] < ranks[i]
        avail.discard(i)
        if ok:
            t = best[2]
            log.append((steps - 1, best[1], i))
            for side in (mpo.SIDE_LEFT, mpo.SIDE_RIGHT):
                if best[1] in (side, mpo.SIDE_BOTH):
                    p = pos[side]                  # logical qubit -> site
                    a, b = p.index(i), p.index(i + 1)
                    p[a], p[b] = i + 1, i
            for nb in (i - 1, i + 1):
                if 0 <= nb < n - 1:
                    avail.add(nb)
    return log, t, pos, steps


@pytest.mark.parametrize("circ,equal,min_accepts", [
    (W.hidden_permutation_mirror(6, 6, 0.0, seed=2), False, 5),
    (W.permutation_only(6, seed=4), False, 2),
    (W.permutation_only(6, seed=1), False, 2),
    (W.random_circuit(6, 10, seed=3), False, 0),     # no swap lowers a rank: rejections only
    (W.permutation_only(5, seed=2), True, 2),
])
def test_sequential_unswap_matches_brute_force(circ, equal, min_accepts):
    """The oracle's sequential unswap log (accepted steps with their step index, side and
    bond), its layouts and its final operator equal a replay of the selection rule on the
    dense operator of the circuit (from the statevector simulator), N <= 6."""
    n = circ.n_qubits
    cfg = mpo.Config(eps=1e-9, chi_max=1 << 20, tau=1e12, unswap_enabled=False,
                     unswap_parallel=False, accept_equal=equal, max_unswap_iter=3 if equal else 20)
    ctr = mpo.Contraction(circ, cfg)
    ctr.run()                                     # M = the whole circuit, nothing unswapped
    # the routed circuit's operator with the sites the router left each qubit on
    pos_l, pos_r = list(ctr.lay[mpo.SIDE_LEFT].pos), list(ctr.lay[mpo.SIDE_RIGHT].pos)
    op = sv.full_operator(circ)
    t0 = sv.operator_to_sites(op, n, pos_l, pos_r) / 2 ** (n / 2)
    cap = cfg.max_unswap_iter * n * 4
    want_log, t_end, pos, _ = _replay_sequential(t0, n, cfg.eps, cfg.chi_max, equal, cap, pos_l, pos_r)
    ctr.unswap_sequential()
    got = [(step, side, bond) for (_, step, side, bond) in ctr.res.unswap_log]
    assert got == want_log
    assert ctr.lay[mpo.SIDE_LEFT].pos == pos[mpo.SIDE_LEFT]
    assert ctr.lay[mpo.SIDE_RIGHT].pos == pos[mpo.SIDE_RIGHT]
    t = ctr.state.B[0]
    for j in range(1, n):
        t = np.tensordot(t, ctr.state.B[j], axes=([-1], [0]))
    assert np.max(np.abs(t.reshape([4] * n) - t_end)) < 1e-12
    assert len(want_log) >= min_accepts


def test_sequential_replay_covers_every_side_and_a_rejection():
    """The hidden-permutation case above exercises all three sides, rejections and the
    re-enabling of neighbours (so a wrong tie order or available-set rule changes its log)."""
    circ = W.hidden_permutation_mirror(6, 6, 0.0, seed=2)
    ctr = mpo.Contraction(circ, mpo.Config(eps=1e-9, chi_max=1 << 20, tau=1e12, unswap_enabled=False))
    ctr.run()
    pos_l, pos_r = list(ctr.lay[mpo.SIDE_LEFT].pos), list(ctr.lay[mpo.SIDE_RIGHT].pos)
    t0 = sv.operator_to_sites(sv.full_operator(circ), 6, pos_l, pos_r) / 8.0
    log, _, _, steps = _replay_sequential(t0, 6, 1e-9, 1 << 20, False, 480, pos_l, pos_r)
    sides = {s for (_, s, _) in log}
    assert len(sides) >= 2
    assert steps > len(log)                       # some steps were rejections
    bonds = [b for (_, _, b) in log]
    assert len(bonds) > len(set(bonds))           # a bond was accepted again after re-enabling


# --- parallel unswapping (App. A.1) replayed on the dense operator -----------------------

_APP_A1_ORDER = [(mpo.SIDE_BOTH, 0), (mpo.SIDE_BOTH, 1), (mpo.SIDE_LEFT, 0), (mpo.SIDE_LEFT, 1),
                 (mpo.SIDE_RIGHT, 0), (mpo.SIDE_RIGHT, 1)]


def _replay_parallel(t, n, eps, chi_max, equal, max_iter, pos_l, pos_r):
    """App. A.1 on the dense site tensor: cycles of six batches (both sides, then left, then
    right; even bonds before odd ones); in a batch every bond of that parity is tried on the
    pre-batch tensor and the swaps whose operator-Schmidt rank drops below the current one (or
    does not grow, in equal mode) are applied (bonds of one parity share no site, so those swaps
    commute and leave each other's cuts alone); a cycle with no acceptance, or max_iter cycles,
    ends the stage."""
    pos = {mpo.SIDE_LEFT: list(pos_l), mpo.SIDE_RIGHT: list(pos_r)}
    log = []
    for it in range(max_iter):
        any_acc = False
        for side, parity in _APP_A1_ORDER:
            bonds = list(range(parity, n - 1, 2))
            old = {b: _count(sv.operator_schmidt_values(t, b), eps, chi_max) for b in bonds}
            new = {b: _count(sv.operator_schmidt_values(_swap_legs(t, n, b, side), b), eps, chi_max)
                   for b in bonds}
            for b in bonds:
                if new[b] <= old[b] if equal else new[b] < old[b]:
                    t = _swap_legs(t, n, b, side)
                    log.append((it, side, b))
                    any_acc = True
                    for s_ in (mpo.SIDE_LEFT, mpo.SIDE_RIGHT):
                        if side in (s_, mpo.SIDE_BOTH):
                            p = pos[s_]
                            x, y = p.index(b), p.index(b + 1)
                            p[x], p[y] = b + 1, b
        if not any_acc:
            break
    return log, t, pos


@pytest.mark.parametrize("circ,equal,min_accepts", [
    (W.hidden_permutation_mirror(6, 6, 0.0, seed=2), False, 3),
    (W.permutation_only(6, seed=4), False, 2),
    (W.permutation_only(6, seed=1), False, 2),
    (W.random_circuit(6, 10, seed=3), False, 0),     # no swap lowers a rank: one empty cycle
    (W.permutation_only(5, seed=2), True, 2),
])
def test_parallel_unswap_matches_brute_force(circ, equal, min_accepts):
    """The oracle's parallel unswap log (cycle, side, bond), its layouts and its final operator
    equal a replay of App. A.1 on the dense operator of the circuit (N <= 6)."""
    n = circ.n_qubits
    cfg = mpo.Config(eps=1e-9, chi_max=1 << 20, tau=1e12, unswap_enabled=False, unswap_parallel=True,
                     accept_equal=equal, max_unswap_iter=3 if equal else 20)
    ctr = mpo.Contraction(circ, cfg)
    ctr.run()
    pos_l, pos_r = list(ctr.lay[mpo.SIDE_LEFT].pos), list(ctr.lay[mpo.SIDE_RIGHT].pos)
    t0 = sv.operator_to_sites(sv.full_operator(circ), n, pos_l, pos_r) / 2 ** (n / 2)
    want_log, t_end, pos = _replay_parallel(t0, n, cfg.eps, cfg.chi_max, equal, cfg.max_unswap_iter,
                                            pos_l, pos_r)
    ctr.unswap_parallel()
    got = [(it, side, bond) for (_, it, side, bond) in ctr.res.unswap_log]
    assert got == want_log
    assert ctr.lay[mpo.SIDE_LEFT].pos == pos[mpo.SIDE_LEFT]
    assert ctr.lay[mpo.SIDE_RIGHT].pos == pos[mpo.SIDE_RIGHT]
    t = ctr.state.B[0]
    for j in range(1, n):
        t = np.tensordot(t, ctr.state.B[j], axes=([-1], [0]))
    assert np.max(np.abs(t.reshape([4] * n) - t_end)) < 1e-12
    assert len(want_log) >= min_accepts


# --- the stall flag (Sec. III.A progress rule) -------------------------------------------

def _schmidt_rank_4x4(g):
    """Operator-Schmidt rank of a two-qubit gate across its two qubits (realigned 4x4)."""
    r = g.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    s = np.linalg.svd(r, compute_uv=False)
    return int(np.sum(s > 1e-9 * s[0]))


def _one_layer_circuit(n, seed):
    """Haar gates on sites (0,1), (2,3), ... then on (1,2), (3,4), ...: all in C_L."""
    rng = W.rng_for(90, seed)
    pairs = [(a, a + 1) for a in range(0, n - 1, 2)] + [(a, a + 1) for a in range(1, n - 1, 2)]
    mats = [W.haar_su4(rng) for _ in pairs]
    return W.Circuit(n, np.array(pairs, np.int32), np.array(mats), 0, np.zeros(0, np.int32),
                     np.zeros((0, 2, 2), np.complex128))


@pytest.mark.parametrize("tau,stalled", [(25, True), (97, False)])
def test_stall_flag_by_construction(tau, stalled):
    """n = 6, C_L = one layer of Haar gates on bonds 0, 2, 4, then one on bonds 1, 3.  After
    the first layer every gate bond has operator-Schmidt rank 4 and no SWAP from either side
    lowers it (checked on each gate), so size(M) = 6 * 16 = 96 whatever unswapping does.
    tau = 25 (just above the identity's 24): the first stage ends at 96 >= tau with a layer
    left, so the run is stalled.  tau = 97: the first stage absorbs both layers and nothing
    is left when the size check runs, so it is not."""
    c = _one_layer_circuit(6, seed=1)
    swap = W.SWAP4
    for g in c.mats[:3]:
        assert min(_schmidt_rank_4x4(x) for x in (g, swap @ g, g @ swap, swap @ g @ swap)) == 4
    r = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=1 << 20, tau=tau))
    assert r.stalled == stalled
    if stalled:
        assert r.trace[0]["size"] == 96 and r.trace[1]["size"] == 96


def test_stall_flag_clears_when_unswapping_brings_size_below_tau():
    """A permutation-only circuit exceeds tau before unswapping and returns to the identity's
    size 4n after it (every bond at 1): not stalled, although the pre-unswap size is >= tau."""
    c = W.permutation_only(8, seed=3, planted=False)
    tau = 4 * 8 + 1
    r = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=256, tau=tau))
    assert any(rec["phase"] == "absorb" and rec["size"] >= tau for rec in r.trace)
    assert r.trace[-1]["size"] == 4 * 8
    assert not r.stalled
    r2 = mpo.contract(c, mpo.Config(eps=1e-12, chi_max=256, tau=tau, unswap_enabled=False))
    assert r2.stalled == any(rec["size"] >= tau for rec in r2.trace[:-1])
