"""Seeded synthetic mirrored circuits (inputs only; none of the contraction method lives here).

These generators stand in for the paper's HQAP benchmark circuits (Sec. III, a 56-qubit
circuit with 1,917 two-qubit gates built as a mirrored U U^dagger block with swap
obfuscation, Sec. I).  The circuit files themselves are not available, so every workload
here is synthesised from a seed with the same structure:

* a brickwork mirror on a line (the unobfuscated case the Middle-MPO attack solves, Sec. I);
* an all-to-all mirror whose two halves are separated by a hidden qubit permutation
  written as innocuous-looking two-qubit gates (the swap obfuscation unswapping removes,
  Sec. II.B.2), with a per-gate perturbation exp(i eps H) on the mirrored half so the
  output is peaked but not exactly a basis state.

Both the oracle and the GPU library consume exactly the arrays produced here: logical
qubit pairs ``pairs[g] = (a, b)`` (gate basis index ``2*x_a + x_b``), FP64 4x4 matrices,
the split index between the right (earlier) and left (later) halves, and a final layer of
one-qubit gates (the planted X^s).  Bit order for bitstrings: ``bits[q]`` is logical qubit
q; a statevector index is ``sum_q bits[q] * 2**q``.

Random numbers: numpy PCG64 seeded by ``SeedSequence(260421908, spawn_key=(family, seed))``.
Haar SU(4) follows Mezzadri (2007): QR of a complex Ginibre matrix with the phases of
R's diagonal moved into Q, then divided by det^(1/4).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ROOT_SEED = 260421908

SWAP4 = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
X2 = np.array([[0, 1], [1, 0]], dtype=np.complex128)


@dataclass
class Circuit:
    """A gate list in time order plus the split point and the final one-qubit layer."""

    n_qubits: int
    pairs: np.ndarray                 # int32 [G, 2] logical qubits, pairs[g, 0] is the MSB of the gate basis
    mats: np.ndarray                  # complex128 [G, 4, 4]
    split_index: int                  # gates[:split] form the right (earlier) half C_R
    oneq_qubits: np.ndarray           # int32 [K] one-qubit gates applied after every two-qubit gate
    oneq_mats: np.ndarray             # complex128 [K, 2, 2]
    planted: np.ndarray | None = None  # uint8 [n] the bitstring s the circuit is built to peak on
    permutation: np.ndarray | None = None  # int32 [n] hidden permutation pi (qubit q -> pi[q])
    meta: dict = field(default_factory=dict)

    @property
    def n_gates(self) -> int:
        return int(self.pairs.shape[0])

    def mats_interleaved(self) -> np.ndarray:
        """[G, 4, 4, 2] float64 (re, im), the layout the C library takes."""
        return np.ascontiguousarray(np.stack([self.mats.real, self.mats.imag], axis=-1))

    def oneq_interleaved(self) -> np.ndarray:
        return np.ascontiguousarray(np.stack([self.oneq_mats.real, self.oneq_mats.imag], axis=-1))


def rng_for(family: int, seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(ROOT_SEED, spawn_key=(family, seed))))


def haar_unitary(rng: np.random.Generator, d: int = 4) -> np.ndarray:
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def haar_su4(rng: np.random.Generator) -> np.ndarray:
    u = haar_unitary(rng, 4)
    det = np.linalg.det(u)
    return u / det ** 0.25


def polar_unitarize(g: np.ndarray) -> np.ndarray:
    """Nearest unitary to g (polar factor), via the FP64 eigendecomposition of g^dagger g."""
    w, v = np.linalg.eigh(g.conj().T @ g)
    return g @ (v * (1.0 / np.sqrt(w))[None, :]) @ v.conj().T


def through_complex64(g: np.ndarray) -> np.ndarray:
    """A gate stored as complex64, read back as FP64 and re-unitarised."""
    return polar_unitarize(g.astype(np.complex64).astype(np.complex128))


def random_traceless_hermitian(rng: np.random.Generator, d: int = 4) -> np.ndarray:
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    h = 0.5 * (z + z.conj().T)
    h = h - np.trace(h) / d * np.eye(d)
    return h / np.max(np.abs(np.linalg.eigvalsh(h)))


def expi_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * eps * w)[None, :]) @ v.conj().T


def relabel_gate(pair, perm):
    return (int(perm[pair[0]]), int(perm[pair[1]]))


def permutation_transpositions(perm: np.ndarray) -> list[tuple[int, int]]:
    """SWAPs (time order) that move the state of qubit q to qubit perm[q].

    A cycle c0 -> c1 -> ... -> c_{L-1} -> c0 is realised by SWAP(c0,c1), SWAP(c0,c2), ...,
    SWAP(c0,c_{L-1}).
    """
    n = len(perm)
    seen = np.zeros(n, dtype=bool)
    out = []
    for start in range(n):
        if seen[start]:
            continue
        cyc = [start]
        seen[start] = True
        q = int(perm[start])
        while q != start:
            cyc.append(q)
            seen[q] = True
            q = int(perm[q])
        for k in range(1, len(cyc)):
            out.append((cyc[0], cyc[k]))
    return out


def _oneq_layer(planted: np.ndarray):
    qs = np.nonzero(planted)[0].astype(np.int32)
    mats = np.repeat(X2[None], len(qs), axis=0)
    return qs, mats


def brickwork_mirror(n: int, layers: int, seed: int = 0) -> Circuit:
    """X^s . U^dagger . U with U a brickwork of Haar SU(4) gates on a line (no permutation).

    U has `layers` layers, alternating even bonds (0,1),(2,3),... and odd bonds.  The
    right half C_R is U; the left half is U^dagger followed by X^s.
    """
    rng = rng_for(1, seed)
    pairs, mats = [], []
    for layer in range(layers):
        for a in range(layer % 2, n - 1, 2):
            pairs.append((a, a + 1))
            mats.append(haar_su4(rng))
    g_half = len(pairs)
    for k in range(g_half - 1, -1, -1):
        pairs.append(pairs[k])
        mats.append(mats[k].conj().T)
    planted = rng.integers(0, 2, size=n).astype(np.uint8)
    oq, om = _oneq_layer(planted)
    return Circuit(n, np.array(pairs, dtype=np.int32), np.array(mats), g_half, oq, om, planted,
                   np.arange(n, dtype=np.int32), {"family": "brickwork_mirror", "layers": layers, "seed": seed})


def hidden_permutation_mirror(n: int, gates_per_half: int, eps_pert: float, seed: int = 0,
                              store_complex64: bool = True, family: int = 2) -> Circuit:
    """X^s . V^dagger . P_pi . U with V = P_pi U P_pi^dagger, so C|0> = |s> when eps_pert = 0.

    * U: `gates_per_half` Haar SU(4) gates on uniformly random distinct pairs (a, b).
    * P_pi: a seeded random permutation written as transpositions; each transposition
      (a, b) becomes the two gates R then SWAP.R^dagger on (a, b) with R Haar, so no SWAP
      appears in the gate list.
    * V^dagger: U's gates relabelled by pi, in reverse time order, adjoint, each
      left-multiplied by exp(i eps_pert H_k) with H_k a random traceless Hermitian of unit
      spectral norm.
    * X^s: a final layer of X gates on the planted bitstring s.
    With store_complex64 the U gates go through complex64 and are re-unitarised in FP64
    before the mirror is built, so the mirror stays exact in FP64.
    """
    rng = rng_for(family, seed)
    cast = through_complex64 if store_complex64 else (lambda g: g)
    u_pairs, u_mats = [], []
    for _ in range(gates_per_half):
        a, b = rng.choice(n, size=2, replace=False)
        u_pairs.append((int(a), int(b)))
        u_mats.append(cast(haar_su4(rng)))
    perm = rng.permutation(n).astype(np.int32)
    p_pairs, p_mats = [], []
    for (a, b) in permutation_transpositions(perm):
        r = cast(haar_su4(rng))
        p_pairs += [(a, b), (a, b)]
        p_mats += [r, SWAP4 @ r.conj().T]
    v_pairs, v_mats = [], []
    for k in range(gates_per_half - 1, -1, -1):
        g = u_mats[k].conj().T
        if eps_pert != 0.0:
            g = expi_hermitian(random_traceless_hermitian(rng), eps_pert) @ g
        v_pairs.append(relabel_gate(u_pairs[k], perm))
        v_mats.append(g)
    planted = rng.integers(0, 2, size=n).astype(np.uint8)
    oq, om = _oneq_layer(planted)
    pairs = np.array(u_pairs + p_pairs + v_pairs, dtype=np.int32)
    mats = np.array(u_mats + p_mats + v_mats)
    split = len(pairs) // 2
    return Circuit(n, pairs, mats, split, oq, om, planted, perm,
                   {"family": "hidden_permutation_mirror", "gates_per_half": gates_per_half,
                    "eps_pert": eps_pert, "seed": seed, "n_perm_gates": len(p_pairs)})


def rzz(theta: float) -> np.ndarray:
    """RZZ(theta) = exp(-i theta/2 Z(x)Z), the trapped-ion native two-qubit gate."""
    a = np.exp(-0.5j * theta)
    return np.diag([a, np.conj(a), np.conj(a), a]).astype(np.complex128)


def haar_su2(rng: np.random.Generator) -> np.ndarray:
    u = haar_unitary(rng, 2)
    return u / np.sqrt(np.linalg.det(u))


_H2 = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
_SDG = np.diag([1.0, -1.0j]).astype(np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _cnot_from_rzz(control_first: bool) -> np.ndarray:
    """CNOT written in the native set: CZ = e^{i pi/4} (S^dagger (x) S^dagger) RZZ(pi/2), with
    Hadamards on the target."""
    cz = np.exp(0.25j * np.pi) * np.kron(_SDG, _SDG) @ rzz(0.5 * np.pi)
    h = np.kron(_I2, _H2) if control_first else np.kron(_H2, _I2)
    return h @ cz @ h


def swap_as_native_gates(rng: np.random.Generator) -> list[np.ndarray]:
    """A SWAP as three two-qubit gates, each one RZZ(pi/2) dressed with one-qubit gates:
    CNOT(a->b) CNOT(b->a) CNOT(a->b) with random SU(2) pairs inserted between them and undone
    in the next gate, so no gate looks like a SWAP or a CNOT.  The product (time order g1, g2,
    g3) is exactly SWAP."""
    c_ab, c_ba = _cnot_from_rzz(True), _cnot_from_rzz(False)
    r1 = np.kron(haar_su2(rng), haar_su2(rng))
    r2 = np.kron(haar_su2(rng), haar_su2(rng))
    return [r1 @ c_ab, r2 @ c_ba @ r1.conj().T, c_ab @ r2.conj().T]


def hqap_like_mirror(n: int, rzz_per_half: int, n_swaps: int, angle_noise: float, seed: int = 0) -> Circuit:
    """A peaked circuit shaped like the HQAP construction the paper attacks (Sec. I, Sec. III:
    RZZ two-qubit gates with one-qubit layers, a U U^dagger mirror, swap insertions, angle
    sweeping, a planted bitstring).  Synthetic: nothing here reconstructs the paper's circuit.

    * U: layers of RZZ(theta) gates on random perfect matchings of the qubits (all-to-all, as on
      a trapped-ion machine), each preceded by Haar SU(2) gates on its two qubits (the one-qubit
      layers, fused into the two-qubit gate); theta uniform in [0.2, pi - 0.2].
    * Swap insertion: a permutation pi made of `n_swaps` transpositions of random qubit pairs,
      each SWAP written as three RZZ-native gates (`swap_as_native_gates`).
    * The mirrored half V^dagger with V = P_pi U P_pi^dagger: U's gates in reverse order,
      relabelled by pi, each inverted with its RZZ angle swept by a Gaussian offset of standard
      deviation `angle_noise` (the peak weight falls roughly as exp(-rzz_per_half
      angle_noise^2 / 4)).
    * X^s: the planted bitstring, last in time.
    The gate list is two-qubit 4x4 matrices (one-qubit gates fused) plus the final X layer."""
    rng = rng_for(15, seed)
    u_pairs, u_mats, u_parts = [], [], []
    while len(u_pairs) < rzz_per_half:
        order = rng.permutation(n)
        for k in range(0, n - 1, 2):
            if len(u_pairs) == rzz_per_half:
                break
            a, b = int(order[k]), int(order[k + 1])
            theta = float(rng.uniform(0.2, np.pi - 0.2))
            dress = np.kron(haar_su2(rng), haar_su2(rng))
            u_pairs.append((a, b))
            u_mats.append(rzz(theta) @ dress)
            u_parts.append((theta, dress))
    perm = np.arange(n, dtype=np.int32)
    p_pairs, p_mats = [], []
    for _ in range(n_swaps):
        a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
        for g in swap_as_native_gates(rng):
            p_pairs.append((a, b))
            p_mats.append(g)
        pa = np.nonzero(perm == a)[0][0]
        pb = np.nonzero(perm == b)[0][0]
        perm[pa], perm[pb] = b, a
    v_pairs, v_mats = [], []
    for k in range(rzz_per_half - 1, -1, -1):
        theta, dress = u_parts[k]
        delta = float(rng.normal(0.0, angle_noise)) if angle_noise > 0 else 0.0
        v_pairs.append(relabel_gate(u_pairs[k], perm))
        v_mats.append(dress.conj().T @ rzz(-theta + delta))
    planted = rng.integers(0, 2, size=n).astype(np.uint8)
    oq, om = _oneq_layer(planted)
    pairs = np.array(u_pairs + p_pairs + v_pairs, dtype=np.int32)
    mats = np.array(u_mats + p_mats + v_mats)
    return Circuit(n, pairs, mats, len(pairs) // 2, oq, om, planted, perm,
                   {"family": "hqap_like_mirror", "rzz_per_half": rzz_per_half, "n_swaps": n_swaps,
                    "angle_noise": angle_noise, "seed": seed})


def random_circuit(n: int, n_gates: int, seed: int = 0, line: bool = False) -> Circuit:
    """A circuit with no mirror structure (Haar gates on random pairs), for checks where
    the MPO must reproduce an arbitrary unitary."""
    rng = rng_for(3, seed)
    pairs, mats = [], []
    for _ in range(n_gates):
        if line:
            a = int(rng.integers(0, n - 1))
            pr = (a, a + 1) if rng.integers(0, 2) == 0 else (a + 1, a)
        else:
            a, b = rng.choice(n, size=2, replace=False)
            pr = (int(a), int(b))
        pairs.append(pr)
        mats.append(haar_su4(rng))
    return Circuit(n, np.array(pairs, dtype=np.int32).reshape(-1, 2), np.array(mats).reshape(-1, 4, 4),
                   n_gates // 2, np.zeros(0, np.int32), np.zeros((0, 2, 2), np.complex128), None, None,
                   {"family": "random", "seed": seed})


def permutation_only(n: int, seed: int = 0, planted: bool = True) -> Circuit:
    """C = X^s . P_pi with P_pi written as a SWAP network over the transpositions of pi."""
    rng = rng_for(4, seed)
    perm = rng.permutation(n).astype(np.int32)
    pairs = permutation_transpositions(perm)
    mats = [SWAP4.copy() for _ in pairs]
    s = rng.integers(0, 2, size=n).astype(np.uint8) if planted else np.zeros(n, np.uint8)
    oq, om = _oneq_layer(s)
    return Circuit(n, np.array(pairs, dtype=np.int32).reshape(-1, 2), np.array(mats).reshape(-1, 4, 4),
                   len(pairs) // 2, oq, om, s, perm, {"family": "permutation_only", "seed": seed})


# --- Uniform random operands for MPO microbenchmarks (a batch of independent two-site updates) ---

def random_right_isometry(rng: np.random.Generator, chi_l: int, chi_r: int) -> np.ndarray:
    """B[chi_l, 4, chi_r] with orthonormal rows (B B^dagger = I), from QR of a Gaussian."""
    z = rng.standard_normal((4 * chi_r, chi_l)) + 1j * rng.standard_normal((4 * chi_r, chi_l))
    q, _ = np.linalg.qr(z)
    return np.ascontiguousarray(q.conj().T.reshape(chi_l, 4, chi_r))


def geometric_spectrum(chi: int, scale: float = 64.0) -> np.ndarray:
    s = np.exp(-np.arange(chi) / scale)
    return s / np.linalg.norm(s)


# --- The named workloads -----------------------------------------------------------------

def workload_line12(seed: int = 0) -> Circuit:
    """n=12 brickwork mirror, 8 layers per half (44 gates per half), complex128."""
    return brickwork_mirror(12, 8, seed)


def workload_unswap28(seed: int = 0) -> Circuit:
    """n=28 all-to-all, 200 Haar gates per half, hidden permutation, eps=0.02, complex64 storage."""
    return hidden_permutation_mirror(28, 200, 0.02, seed, store_complex64=True)


def workload_precision36(seed: int = 0) -> Circuit:
    """n=36 all-to-all, 400 gates per half, hidden permutation, eps=0.03."""
    return hidden_permutation_mirror(36, 400, 0.03, seed, store_complex64=True)


def saturated_bond_dims(n: int, chi_max: int) -> list[int]:
    """[1, 4, 16, ..., chi_max, ..., 16, 4, 1]: every bond at min(chi_max, 4^distance)."""
    chi = [1] * (n + 1)
    for b in range(n - 1):
        chi[b + 1] = min(chi_max, 4 ** min(b + 1, n - 1 - b))
    return chi


def peaked_saturated_state(n: int, chi_max: int, seed: int = 0, delta: float = 0.02):
    """A seeded MPO in the shape the contraction reaches on the perturbed hidden-permutation
    workloads (every interior bond at chi_max), written as right-isometric site tensors
    B_j[chi_{j-1}, 4, chi_j] (p = 2*out + in) and bond spectra.

    Row 0 of every site is sqrt(1-delta) times the identity component (out = in, right bond
    index 0) plus sqrt(delta) times a random unit direction orthogonal to it; the other rows
    complete an orthonormal set.  The operator is thus the identity plus an O(delta) part on
    every site: its output on |0...0> is peaked on 0...0.  Spectra: 1 followed by
    sqrt(delta) exp(-k/64), normalised."""
    rng = rng_for(11, seed)
    chi = saturated_bond_dims(n, chi_max)
    B = []
    for j in range(n):
        cl, cr = chi[j], chi[j + 1]
        d = 4 * cr
        e_id = np.zeros(d, dtype=np.complex128)
        e_id[0 * cr + 0] = e_id[3 * cr + 0] = 1.0 / np.sqrt(2.0)
        w = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        w -= e_id * np.vdot(e_id, w)
        w /= np.linalg.norm(w)
        row0 = np.sqrt(1.0 - delta) * e_id + np.sqrt(delta) * w
        z = rng.standard_normal((d, cl)) + 1j * rng.standard_normal((d, cl))
        z[:, 0] = row0
        q, r = np.linalg.qr(z)
        q = q * (np.diag(r) / np.abs(np.diag(r)))[None, :]     # column 0 equals row0 exactly
        B.append(np.ascontiguousarray(q.conj().T.reshape(cl, 4, cr)))
    lam = []
    for b in range(n - 1):
        k = chi[b + 1]
        s = np.concatenate([[1.0], np.sqrt(delta) * np.exp(-np.arange(1, k) / 64.0)])
        lam.append(s / np.linalg.norm(s))
    return B, lam


# --- Several circuits at once (batching) and request streams (serving) ---------------------

def circuit_mix(count: int, seed: int = 0, n_range=(8, 12), gates_range=(12, 24),
                pert_range=(0.0, 0.04)) -> list[Circuit]:
    """`count` independent hidden-permutation mirrors, each with its own qubit count, gate
    count per half and perturbation drawn uniformly from the given ranges (inclusive for
    the integers), its own hidden permutation and planted bitstring."""
    rng = rng_for(13, seed)
    out = []
    for k in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        g = int(rng.integers(gates_range[0], gates_range[1] + 1))
        e = float(rng.uniform(pert_range[0], pert_range[1]))
        out.append(hidden_permutation_mirror(n, g, e, seed=100000 + 1000 * seed + k))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream of `count` requests at `rate` per
    second: cumulative sums of exponential gaps."""
    rng = rng_for(14, seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
