"""Brute-force statevector and full-operator simulation (pins for the MPO oracle).

TEST INFRASTRUCTURE ONLY.  This is the definition the MPO contraction approximates: the
circuit applied gate by gate to |0...0> (Algorithm 1's Ensure clause: an MPS of C|0>^N).
Bit order: index = sum_q x_q 2^q; gate basis index = 2 x_a + x_b for pair (a, b).
"""
from __future__ import annotations

import numpy as np


def _axis(n: int, q: int) -> int:
    return n - 1 - q          # C-order reshape puts qubit n-1 on axis 0


def apply_2q(psi: np.ndarray, n: int, a: int, b: int, g: np.ndarray) -> np.ndarray:
    t = psi.reshape([2] * n)
    ax_a, ax_b = _axis(n, a), _axis(n, b)
    t = np.tensordot(g.reshape(2, 2, 2, 2), t, axes=([2, 3], [ax_a, ax_b]))
    t = np.moveaxis(t, [0, 1], [ax_a, ax_b])
    return t.reshape(-1)


def apply_1q(psi: np.ndarray, n: int, q: int, g: np.ndarray) -> np.ndarray:
    t = psi.reshape([2] * n)
    ax = _axis(n, q)
    t = np.tensordot(g, t, axes=([1], [ax]))
    t = np.moveaxis(t, 0, ax)
    return t.reshape(-1)


def run_circuit(circuit, psi0: np.ndarray | None = None) -> np.ndarray:
    n = circuit.n_qubits
    if psi0 is None:
        psi = np.zeros(2 ** n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = psi0.astype(np.complex128).copy()
    for g in range(circuit.n_gates):
        a, b = int(circuit.pairs[g, 0]), int(circuit.pairs[g, 1])
        psi = apply_2q(psi, n, a, b, circuit.mats[g])
    for q, g2 in zip(circuit.oneq_qubits, circuit.oneq_mats):
        psi = apply_1q(psi, n, int(q), g2)
    return psi


def full_operator(circuit) -> np.ndarray:
    """The 2^n x 2^n unitary of the circuit (columns = images of basis states), n <= 10."""
    n = circuit.n_qubits
    d = 2 ** n
    out = np.empty((d, d), dtype=np.complex128)
    for k in range(d):
        e = np.zeros(d, dtype=np.complex128)
        e[k] = 1.0
        out[:, k] = run_circuit(circuit, e)
    return out


def operator_to_sites(op: np.ndarray, n: int, out_site_of_qubit, in_site_of_qubit) -> np.ndarray:
    """Reshape a 2^n x 2^n operator into the site-ordered tensor T[p_0, ..., p_{n-1}] with
    p_j = 2 o_j + i_j, where o_j is the output bit of the qubit at out-site j and i_j the
    input bit of the qubit at in-site j."""
    t = op.reshape([2] * (2 * n))      # axes: out qubits n-1..0, then in qubits n-1..0
    perm = []
    out_qubit_at = [0] * n
    in_qubit_at = [0] * n
    for q in range(n):
        out_qubit_at[out_site_of_qubit[q]] = q
        in_qubit_at[in_site_of_qubit[q]] = q
    for j in range(n):
        perm.append(_axis(n, out_qubit_at[j]))
        perm.append(n + _axis(n, in_qubit_at[j]))
    return np.transpose(t, perm).reshape([4] * n)


def operator_schmidt_values(t: np.ndarray, cut: int) -> np.ndarray:
    """Normalised operator-Schmidt values of the site tensor across bond `cut` (sites
    0..cut | cut+1..n-1): singular values of the reshaped tensor scaled to sum s^2 = 1."""
    n = t.ndim
    m = t.reshape(4 ** (cut + 1), 4 ** (n - cut - 1))
    s = np.linalg.svd(m, compute_uv=False)
    return s / np.linalg.norm(s)
