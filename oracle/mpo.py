"""FP64 oracle: middle-out MPO contraction with greedy unswapping (Algorithm 1 of the paper).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Plain numpy/scipy, FP64, no
blocking or fusion beyond what the method states.

Representation (the reading used throughout; the paper says only "canonical form via SVD",
Sec. II.B.1 / Algorithm 1 "Compress M to canonical form"):
  * The MPO M (Sec. II.A, identity at the midpoint) is stored as a local-dimension-4 MPS
    |M>> over per-site index p = 2*o + i (o = output leg, i = input leg), Frobenius-
    normalised, in Vidal form with Hastings' update: right-canonical site tensors
    B[j] of shape (chi_{j-1}, 4, chi_j) and bond spectra lam[j] (bond j joins sites j, j+1).
    |M>> = B[0] B[1] ... B[N-1]; lam[j] are the normalised operator-Schmidt values.
  * Absorbing a gate g from the left (M <- g M) acts on the out-legs, a gate h from the
    right (M <- M h) on the in-legs; on |M>> both are one 16x16 operator on (p_j, p_{j+1}).
  * layout_l / layout_r map logical qubit -> site for the left / right circuits.  A SWAP
    taken into M from one side permutes that side's layout (this is how the permutations
    P_L, P_R of Eq. 1 are recorded, and how rewiring reindexes the remaining circuit).
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

SWAP4 = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
I4 = np.eye(4, dtype=np.complex128)

SIDE_LEFT, SIDE_RIGHT, SIDE_BOTH = 0, 1, 2
SIDE_NAMES = {SIDE_LEFT: "left", SIDE_RIGHT: "right", SIDE_BOTH: "both"}
# App. A.1: the six (side, parity) combinations cycled in this order.
PARALLEL_ORDER = [(SIDE_BOTH, 0), (SIDE_BOTH, 1), (SIDE_LEFT, 0), (SIDE_LEFT, 1),
                  (SIDE_RIGHT, 0), (SIDE_RIGHT, 1)]


@dataclass
class Config:
    """Hyperparameters of App. A.4 (SVD cutoff, chi_max, tau, max unswap iterations,
    acceptance mode) plus the unswap variant (App. A.1 parallel vs Algorithm 1 sequential)."""

    eps: float = 1e-10
    chi_max: int = 256
    tau: float = 1e6
    max_unswap_iter: int = 20
    accept_equal: bool = False      # App. A.2 non-strict acceptance
    unswap_parallel: bool = True    # App. A.1 parallel swap selection
    unswap_enabled: bool = True     # False = the plain Middle-MPO attack (Sec. I)
    side_adaptive: bool = False     # App. A.3 adaptive side selection (else alternate L, R)
    recanonicalise: bool = True     # Algorithm 1 "compress M to canonical form" after each
                                    # absorption step and before the projection


def two_site_operator(g: np.ndarray | None = None, h: np.ndarray | None = None) -> np.ndarray:
    """16x16 operator on (p1, p2), p = 2*o + i, for M <- g M h (Sec. II.B.1 absorption).

    g acts on the out-legs (o1, o2) with basis index 2*o1 + o2; h on the in-legs, with
    M'[o, i] = sum_i' M[o, i'] h[i', i].  Row index 4*p1 + p2 (new), column 4*p1' + p2'.
    """
    g = I4 if g is None else g
    h = I4 if h is None else h
    g4 = g.reshape(2, 2, 2, 2)      # [o1, o2, o1', o2']
    h4 = h.reshape(2, 2, 2, 2)      # [i1', i2', i1, i2]
    u = np.einsum("abcd,efgh->agbhcedf", g4, h4)   # [o1, i1, o2, i2, o1', i1', o2', i2']
    return u.reshape(16, 16)


def swap_operator(side: int) -> np.ndarray:
    """The 16x16 operator of a SWAP taken into M from the left, right or both sides
    (Algorithm 1, ApplySwap)."""
    if side == SIDE_LEFT:
        return two_site_operator(SWAP4, None)
    if side == SIDE_RIGHT:
        return two_site_operator(None, SWAP4)
    return two_site_operator(SWAP4, SWAP4)


def truncation_count(s: np.ndarray, eps: float, chi_max: int) -> int:
    """Number of singular values kept: s_k > eps * s_0 (relative cutoff, Sec. II.B.1 and
    App. A.4), at least 1, at most chi_max.  s is sorted descending."""
    if s.size == 0 or s[0] <= 0.0:
        return 1
    k = int(np.count_nonzero(s > eps * s[0]))
    return max(1, min(k, chi_max))


@dataclass
class UpdateRecord:
    side: int      # 0 left / 1 right / 2 both
    bond: int
    kind: int      # 0 routing swap, 1 gate, 2 unswap trial accepted
    gate: int      # gate index into the circuit's list, -1 for swaps
    chi: int = 0   # bond dimension after the update


@dataclass
class Trial:
    count: int
    s: np.ndarray
    vh: np.ndarray
    theta0: np.ndarray
    chi_l: int
    chi_r: int


class MPOState:
    """The MPO M in Vidal/Hastings form (see module docstring)."""

    def __init__(self, n: int):
        self.n = n
        b = np.zeros((1, 4, 1), dtype=np.complex128)
        b[0, 0, 0] = b[0, 3, 0] = 1.0 / math.sqrt(2.0)   # identity on one qubit, Frobenius norm 1
        self.B = [b.copy() for _ in range(n)]             # Algorithm 1: M <- I^{(x)N}, bond dimension 1
        self.lam = [np.ones(1) for _ in range(n - 1)]

    def chi(self, j: int) -> int:
        return int(self.B[j].shape[2])

    def bond_dims(self) -> list[int]:
        return [self.chi(j) for j in range(self.n - 1)]

    def size(self) -> int:
        """size(M): total number of tensor elements of the MPO (Sec. II.B.1)."""
        return int(sum(b.size for b in self.B))

    def lam_left(self, j: int) -> np.ndarray:
        return self.lam[j - 1] if j > 0 else np.ones(1)

    # -- Sec. II.B.1: contract the two-qubit gate with the two site tensors, then SVD ------
    def trial(self, j: int, u16: np.ndarray, cfg: Config) -> Trial:
        """Merge sites j, j+1, apply the 16x16 operator, factorise the (4 chi_l) x (4 chi_r)
        bond matrix by SVD and count the singular values above the cutoff."""
        bl, br = self.B[j], self.B[j + 1]
        chi_l, chi_r = bl.shape[0], br.shape[2]
        theta0 = np.einsum("lpm,mqr->lpqr", bl, br)                              # merge
        theta0 = np.einsum("PQpq,lpqr->lPQr", u16.reshape(4, 4, 4, 4), theta0)   # gate
        theta = self.lam_left(j)[:, None, None, None] * theta0
        x = theta.reshape(4 * chi_l, 4 * chi_r)                                  # reshape
        _, s, vh = scipy.linalg.svd(x, full_matrices=False, lapack_driver="gesvd")  # factorise
        k = truncation_count(s, cfg.eps, cfg.chi_max)
        return Trial(k, s, vh, theta0.reshape(4 * chi_l, 4 * chi_r), chi_l, chi_r)

    def commit(self, j: int, t: Trial) -> None:
        """Truncate to t.count values, renormalise sum s^2 = 1 and split (Hastings form:
        B[j+1] <- V^dagger, B[j] <- Theta_without_lambda V / |s_kept|, lam[j] <- s_kept)."""
        k = t.count
        vh = t.vh[:k]
        nrm = float(np.linalg.norm(t.s[:k]))
        self.B[j + 1] = np.ascontiguousarray(vh.reshape(k, 4, t.chi_r))
        self.B[j] = np.ascontiguousarray((t.theta0 @ vh.conj().T / nrm).reshape(t.chi_l, 4, k))
        self.lam[j] = t.s[:k] / nrm

    def apply(self, j: int, u16: np.ndarray, cfg: Config) -> int:
        t = self.trial(j, u16, cfg)
        self.commit(j, t)
        return t.count

    def recanonicalise(self, cfg: Config) -> None:
        """Algorithm 1, "compress M to canonical form via SVD with eps": a left-to-right QR
        sweep leaves every site left-orthonormal and carries the rest to the right; a
        right-to-left SVD sweep then makes every site right-canonical (B_j = V^dagger), reads
        the bond's Schmidt values with everything to its left orthonormal, applies the cutoff
        (s_k > eps s_0, at least 1, at most chi_max) and carries U S to the left.  Afterwards
        the stored B_j and lam_j are the Vidal/Hastings form of the current operator (under
        truncation the two-site updates drift away from it).  |M>> is renormalised."""
        n = self.n
        B = [b.copy() for b in self.B]
        for j in range(n - 1):
            cl, _, cr = B[j].shape
            q, r = np.linalg.qr(B[j].reshape(cl * 4, cr))
            B[j] = q.reshape(cl, 4, q.shape[1])
            B[j + 1] = np.einsum("ab,bpc->apc", r, B[j + 1])
        for j in range(n - 1, 0, -1):
            cl, _, cr = B[j].shape
            u, s, vh = scipy.linalg.svd(B[j].reshape(cl, 4 * cr), full_matrices=False, lapack_driver="gesvd")
            k = truncation_count(s, cfg.eps, cfg.chi_max)
            B[j] = np.ascontiguousarray(vh[:k].reshape(k, 4, cr))
            self.lam[j - 1] = s[:k] / np.linalg.norm(s[:k])
            B[j - 1] = np.einsum("apb,bc->apc", B[j - 1], u[:, :k] * s[None, :k])
        B[0] = B[0] / np.linalg.norm(B[0])
        self.B = B

    def apply_one_site(self, j: int, g2: np.ndarray, side: int) -> None:
        """A one-qubit gate on the out-legs (side left) or in-legs (side right) of site j;
        unitary on one site, so the canonical form is unchanged."""
        b = self.B[j].reshape(self.B[j].shape[0], 2, 2, self.B[j].shape[2])   # [l, o, i, r]
        if side == SIDE_LEFT:
            b = np.einsum("ab,lbir->lair", g2, b)
        else:
            b = np.einsum("lobr,ba->loar", b, g2)
        self.B[j] = np.ascontiguousarray(b.reshape(self.B[j].shape))


class Layout:
    """Logical qubit <-> site maps for one side (the permutation P_L or P_R of Eq. 1)."""

    def __init__(self, n: int):
        self.pos = list(range(n))     # logical qubit -> site
        self.site = list(range(n))    # site -> logical qubit

    def swap_sites(self, j: int) -> None:
        a, b = self.site[j], self.site[j + 1]
        self.site[j], self.site[j + 1] = b, a
        self.pos[a], self.pos[b] = j + 1, j


def layers_from(order: list[int], pairs: np.ndarray) -> list[list[int]]:
    """Greedy as-soon-as-possible layering of gates in absorption order (the paper's
    "innermost layer", Algorithm 1, for circuits without a given layer structure): a gate
    goes one layer past the last layer that used either of its qubits."""
    last: dict[int, int] = {}
    layers: list[list[int]] = []
    for g in order:
        a, b = int(pairs[g, 0]), int(pairs[g, 1])
        lay = max(last.get(a, -1), last.get(b, -1)) + 1
        if lay == len(layers):
            layers.append([])
        layers[lay].append(g)
        last[a] = last[b] = lay
    return layers


@dataclass
class Result:
    state: MPOState
    layout_l: Layout
    layout_r: Layout
    plan: list[UpdateRecord] = field(default_factory=list)
    unswap_log: list[tuple[int, int, int, int]] = field(default_factory=list)  # (stage, iter, side, bond)
    trace: list[dict] = field(default_factory=list)
    stalled: bool = False
    n_updates: int = 0
    n_trials: int = 0
    sides: list[int] = field(default_factory=list)     # App. A.3: side absorbed per step


class Contraction:
    """Algorithm 1: transpile (route), split, absorb from both sides, unswap, rewire."""

    def __init__(self, circuit, cfg: Config):
        self.c = circuit
        self.cfg = cfg
        n = circuit.n_qubits
        self.n = n
        self.state = MPOState(n)
        self.lay = {SIDE_LEFT: Layout(n), SIDE_RIGHT: Layout(n)}
        g = circuit.n_gates
        split = circuit.split_index
        # C_L (later half) in time order, C_R (earlier half) in reverse time order: the
        # innermost layers are adjacent to M (Sec. II.A).
        self.left_layers = layers_from(list(range(split, g)), circuit.pairs)
        self.right_layers = layers_from(list(range(split - 1, -1, -1)), circuit.pairs)
        self.left_cursor = 0
        self.right_cursor = 0
        self.oneq_done = len(circuit.oneq_qubits) == 0
        self.res = Result(self.state, self.lay[SIDE_LEFT], self.lay[SIDE_RIGHT])
        self.stage = 0

    # -- Sec. II.A: transpile to a line; the router here is the deterministic reading ----
    def _route_and_apply(self, side: int, gidx: int) -> None:
        lay = self.lay[side]
        a, b = int(self.c.pairs[gidx, 0]), int(self.c.pairs[gidx, 1])
        p, q = lay.pos[a], lay.pos[b]
        swap_op = swap_operator(side)
        while abs(p - q) > 1:           # move the first-listed qubit one site toward the second
            j = p if p < q else p - 1
            chi = self.state.apply(j, swap_op, self.cfg)
            lay.swap_sites(j)
            self.res.plan.append(UpdateRecord(side, j, 0, -1, chi))
            self.res.n_updates += 1
            p = lay.pos[a]
        gate = self.c.mats[gidx]
        if p > q:                        # qubit order reversed relative to the sites
            gate = SWAP4 @ gate @ SWAP4
        j = min(p, q)
        u16 = two_site_operator(gate, None) if side == SIDE_LEFT else two_site_operator(None, gate)
        chi = self.state.apply(j, u16, self.cfg)
        self.res.plan.append(UpdateRecord(side, j, 1, gidx, chi))
        self.res.n_updates += 1

    def _absorb_left_layer(self) -> None:
        if self.left_cursor < len(self.left_layers):
            for gidx in self.left_layers[self.left_cursor]:
                self._route_and_apply(SIDE_LEFT, gidx)
            self.left_cursor += 1
        elif not self.oneq_done:
            # the one-qubit layer X^s is the outermost (last in time) part of C_L
            for q, g2 in zip(self.c.oneq_qubits, self.c.oneq_mats):
                self.state.apply_one_site(self.lay[SIDE_LEFT].pos[int(q)], g2, SIDE_LEFT)
            self.oneq_done = True

    def _absorb_right_layer(self) -> None:
        if self.right_cursor < len(self.right_layers):
            for gidx in self.right_layers[self.right_cursor]:
                self._route_and_apply(SIDE_RIGHT, gidx)
            self.right_cursor += 1

    def _save(self):
        st = self.state
        return ([b.copy() for b in st.B], [l.copy() for l in st.lam],
                {k: (list(v.pos), list(v.site)) for k, v in self.lay.items()},
                self.left_cursor, self.right_cursor, self.oneq_done, list(self.res.plan), self.res.n_updates)

    def _load(self, saved) -> None:
        B, lam, lays, lc, rc, oq, plan, nup = saved
        self.state.B = [b.copy() for b in B]
        self.state.lam = [l.copy() for l in lam]
        for k, (pos, site) in lays.items():
            self.lay[k].pos[:] = pos
            self.lay[k].site[:] = site
        self.left_cursor, self.right_cursor, self.oneq_done = lc, rc, oq
        self.res.plan[:] = plan
        self.res.n_updates = nup

    def _absorb_step_adaptive(self) -> int:
        """App. A.3: absorb the next layer of C_L and, separately, of C_R into copies of M and
        keep the one with the smaller size(M).  Reading: ties go to the left (Algorithm 1
        absorbs the left side first); when one side has no layer left the other is absorbed;
        the one-qubit layer X^s counts as the last layer of C_L.  Only the kept absorption
        appears in the plan.  Returns the side absorbed."""
        can_l = self.left_cursor < len(self.left_layers) or not self.oneq_done
        can_r = self.right_cursor < len(self.right_layers)
        if not can_r:
            self._absorb_left_layer()
            return SIDE_LEFT
        if not can_l:
            self._absorb_right_layer()
            return SIDE_RIGHT
        base = self._save()
        self._absorb_left_layer()
        size_l = self.state.size()
        after_l = self._save()
        self._load(base)
        self._absorb_right_layer()
        if size_l <= self.state.size():
            self._load(after_l)
            return SIDE_LEFT
        return SIDE_RIGHT

    def gates_absorbed(self) -> int:
        """Two-qubit gates of C absorbed so far (both sides; the telemetry of Fig. 3)."""
        return (sum(len(l) for l in self.left_layers[:self.left_cursor])
                + sum(len(l) for l in self.right_layers[:self.right_cursor]))

    def layers_remain(self) -> bool:
        return (self.left_cursor < len(self.left_layers) or not self.oneq_done
                or self.right_cursor < len(self.right_layers))

    # -- Sec. II.B.2 unswapping ------------------------------------------------------------
    def _accepts(self, new: int, old: int) -> bool:
        return new <= old if self.cfg.accept_equal else new < old

    def _record_swap(self, side: int, bond: int) -> None:
        if side in (SIDE_LEFT, SIDE_BOTH):
            self.lay[SIDE_LEFT].swap_sites(bond)
        if side in (SIDE_RIGHT, SIDE_BOTH):
            self.lay[SIDE_RIGHT].swap_sites(bond)

    def unswap_parallel(self) -> int:
        """App. A.1: for each (side, parity) in the fixed order, try the swap on every bond
        of that parity at once (the bonds are disjoint, so every trial reads the pre-batch
        state), keep those that reduce the bond dimension; stop after a full cycle with no
        reduction or after max_unswap_iter cycles.

        Pinned: trial counts equal brute-force operator-Schmidt ranks, strict acceptance lowers
        the total bond dimension, permutation-only circuits end at dimension 1 with the
        permutation in the layouts, the operator is unchanged, and the log, layouts and final
        operator equal a replay of this rule on the dense operator (N <= 6).  The accepted
        sequence on perturbed circuits beyond that size: parity unpinned (no closed form;
        compared with the GPU only)."""
        st = self.state
        accepted_total = 0
        for it in range(self.cfg.max_unswap_iter):
            any_acc = False
            for side, parity in PARALLEL_ORDER:
                op = swap_operator(side)
                bonds = list(range(parity, self.n - 1, 2))
                trials = {i: st.trial(i, op, self.cfg) for i in bonds}
                self.res.n_trials += len(bonds)
                for i in bonds:
                    if self._accepts(trials[i].count, st.chi(i)):
                        st.commit(i, trials[i])
                        self._record_swap(side, i)
                        self.res.unswap_log.append((self.stage, it, side, i))
                        self.res.plan.append(UpdateRecord(side, i, 2, -1, trials[i].count))
                        any_acc = True
                        accepted_total += 1
            if not any_acc:
                break
        return accepted_total

    def unswap_sequential(self) -> int:
        """Algorithm 1 unswapping: take the available bond with the largest dimension
        (smallest index on ties), try left, right and both; accept the smallest resulting
        dimension (ties in that side order) if it reduces the bond; update the available set.

        Pinned on permutation-only circuits (dimension 1, permutation in the layouts) and, for
        N <= 6, step by step against a replay of this selection rule on the dense operator from
        the statevector simulator (bond, side, acceptance, layouts, final operator).  The
        accepted sequence on perturbed circuits at scale: parity unpinned, as for the parallel
        variant."""
        st = self.state
        avail = set(range(self.n - 1))
        accepted_total = 0
        cap = self.cfg.max_unswap_iter * max(self.n, 1) * 4
        steps = 0
        while avail and steps < cap:
            steps += 1
            i = min(avail, key=lambda j: (-st.chi(j), j))
            trials = [st.trial(i, swap_operator(side), self.cfg) for side in (SIDE_LEFT, SIDE_RIGHT, SIDE_BOTH)]
            self.res.n_trials += 3
            best = min(range(3), key=lambda k: (trials[k].count, k))
            if self._accepts(trials[best].count, st.chi(i)):
                st.commit(i, trials[best])
                self._record_swap(best, i)
                self.res.unswap_log.append((self.stage, steps - 1, best, i))
                self.res.plan.append(UpdateRecord(best, i, 2, -1, trials[best].count))
                accepted_total += 1
                avail.discard(i)
                for nb in (i - 1, i + 1):
                    if 0 <= nb < self.n - 1:
                        avail.add(nb)
            else:
                avail.discard(i)
        return accepted_total

    def run(self) -> Result:
        """Algorithm 1 main loop.  Reading for the stall case (Sec. III.A notes the method
        can stall): each outer iteration absorbs at least one layer pair; if size(M) is still
        >= tau after unswapping, the result is flagged stalled.  Pinned on circuits whose size
        after each stage is fixed by construction (stalled, not stalled because nothing is left,
        not stalled because unswapping brought the size under tau)."""
        st, cfg = self.state, self.cfg
        while self.layers_remain():
            first = True
            while (first or st.size() < cfg.tau) and self.layers_remain():
                if cfg.side_adaptive:
                    self.res.sides.append(self._absorb_step_adaptive())
                else:
                    self._absorb_left_layer()
                    self._absorb_right_layer()
                if cfg.recanonicalise:
                    st.recanonicalise(cfg)
                first = False
            self.res.trace.append({"phase": "absorb", "stage": self.stage, "size": st.size(),
                                   "max_chi": max(st.bond_dims()) if self.n > 1 else 1,
                                   "updates": self.res.n_updates, "gates": self.gates_absorbed(),
                                   "accepted": 0})
            accepted = 0
            if cfg.unswap_enabled and self.n > 1:
                if cfg.unswap_parallel:
                    accepted = self.unswap_parallel()
                else:
                    accepted = self.unswap_sequential()
            if st.size() >= cfg.tau and self.layers_remain():
                self.res.stalled = True
            self.res.trace.append({"phase": "unswap", "stage": self.stage, "size": st.size(),
                                   "max_chi": max(st.bond_dims()) if self.n > 1 else 1,
                                   "updates": self.res.n_updates, "gates": self.gates_absorbed(),
                                   "accepted": accepted})
            self.stage += 1
            # Rewiring (Sec. II.B.3): the remaining gates are routed with the current
            # layouts, which already hold P_L and P_R; nothing else changes.
        return self.res


def contract(circuit, cfg: Config | None = None) -> Result:
    return Contraction(circuit, cfg or Config()).run()


# -- Sec. II.C: apply M to |0...0>, then sample / find the peak --------------------------

@dataclass
class OutputMPS:
    A: list            # A[j] of shape (chi_{j-1}, 2, chi_j): B[j] with the in-leg set to 0
    env: list          # env[j] = right environment of sites j..N-1, (chi_{j-1} x chi_{j-1})
    norm2: float       # <psi|psi> for the Frobenius-normalised MPO: Z = env[0]
    site_of_qubit: list  # layout_l.pos: logical qubit -> site of the output leg
    n: int


def project_zero(res: Result) -> OutputMPS:
    """Algorithm 1 final step: apply M to |0...0> (in-legs set to 0, p = 2*o + 0), then the
    right environments env[j] = sum_sigma A_j^sigma env[j+1] A_j^sigma^dagger that give
    every prefix marginal.  (With recanonicalisation the last absorption step already left M
    in canonical form.)"""
    st = res.state
    n = st.n
    A = [np.ascontiguousarray(st.B[j][:, 0::2, :]) for j in range(n)]
    env = [None] * (n + 1)
    env[n] = np.ones((1, 1), dtype=np.complex128)
    for j in range(n - 1, -1, -1):
        e = np.zeros((A[j].shape[0], A[j].shape[0]), dtype=np.complex128)
        for sig in range(2):
            a = A[j][:, sig, :]
            e += a @ env[j + 1] @ a.conj().T
        env[j] = e
    return OutputMPS(A, env, float(env[0][0, 0].real), list(res.layout_l.pos), n)


def site_bits_to_logical(mps: OutputMPS, site_bits) -> np.ndarray:
    return np.array([site_bits[mps.site_of_qubit[q]] for q in range(mps.n)], dtype=np.uint8)


def logical_to_site_bits(mps: OutputMPS, bits) -> list[int]:
    y = [0] * mps.n
    for q in range(mps.n):
        y[mps.site_of_qubit[q]] = int(bits[q])
    return y


def prefix_marginal(mps: OutputMPS, v: np.ndarray, j: int) -> float:
    """Normalised probability of a prefix whose left vector after sites 0..j-1 is v."""
    return float((v @ mps.env[j] @ v.conj()).real) / mps.norm2


def extract_peak(mps: OutputMPS, max_expansions: int = 200000):
    """argmax_x |<x|C|0>|^2 by best-first search over site prefixes ordered by the prefix
    marginal (an upper bound on every completion).  The first complete string popped is
    the exact argmax.  Returns (logical bits, normalised p_peak, raw p = 2^n |<s|M_norm|0>|^2,
    expansions)."""
    n = mps.n
    counter = 0
    heap = [(-1.0, (), counter, np.ones(1, dtype=np.complex128))]
    expansions = 0
    while heap:
        negm, prefix, _, v = heapq.heappop(heap)
        if len(prefix) == n:
            p_norm = -negm
            return site_bits_to_logical(mps, prefix), p_norm, p_norm * mps.norm2, expansions
        expansions += 1
        if expansions > max_expansions:
            raise RuntimeError("peak search exceeded the expansion cap (not peaked)")
        j = len(prefix)
        for sig in (0, 1):
            w = v @ mps.A[j][:, sig, :]
            m = prefix_marginal(mps, w, j + 1)
            counter += 1
            heapq.heappush(heap, (-m, prefix + (sig,), counter, w))
    raise RuntimeError("empty search")


def splitmix64(seed: int, counter: int) -> int:
    """SplitMix64 (Steele, Lea, Flood 2014; Vigna's public-domain reference) evaluated at
    state seed + (counter + 1) * golden-gamma, as a counter-based generator.  Pinned to the
    generator's published outputs (first five from seed 1234567; bucket counts from seed
    987654321)."""
    m = (1 << 64) - 1
    z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def uniforms(seed: int, n_samples: int, n: int) -> np.ndarray:
    """u[s][j] in [0, 1): the top 53 bits of splitmix64(seed, s*n + j) times 2^-53."""
    u = np.empty((n_samples, n))
    for s in range(n_samples):
        for j in range(n):
            u[s, j] = (splitmix64(seed, s * n + j) >> 11) * (1.0 / 9007199254740992.0)
    return u


def sample(mps: OutputMPS, u: np.ndarray) -> np.ndarray:
    """Sec. II.C: sweep the sites left to right and draw each bit from its conditional
    given the bits already drawn: bit = 1 iff u >= P(0 | prefix).  Returns logical bits."""
    n = mps.n
    out = np.zeros((u.shape[0], n), dtype=np.uint8)
    for s in range(u.shape[0]):
        v = np.ones(1, dtype=np.complex128)
        bits = []
        for j in range(n):
            w = [v @ mps.A[j][:, sig, :] for sig in (0, 1)]
            p = [float((wi @ mps.env[j + 1] @ wi.conj()).real) for wi in w]
            p0 = p[0] / (p[0] + p[1])
            bit = 1 if u[s, j] >= p0 else 0
            bits.append(bit)
            v = w[bit] / math.sqrt(p[bit])
        out[s] = site_bits_to_logical(mps, bits)
    return out


def amplitudes(mps: OutputMPS, bits: np.ndarray) -> np.ndarray:
    """<x|C|0> = 2^{n/2} prod_j A_j^{y_j}, y = x mapped to sites (the MPO is stored with
    Frobenius norm 1 instead of 2^{n/2})."""
    n = mps.n
    out = np.zeros(bits.shape[0], dtype=np.complex128)
    for k in range(bits.shape[0]):
        y = logical_to_site_bits(mps, bits[k])
        v = np.ones(1, dtype=np.complex128)
        for j in range(n):
            v = v @ mps.A[j][:, y[j], :]
        out[k] = v[0] * 2.0 ** (n / 2)
    return out
