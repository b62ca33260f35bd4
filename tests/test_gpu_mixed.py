"""Mixed-precision path (merge as complex 3xTF32 on tcgen05 tensor cores, FP32 accumulation;
factorisation, truncation and split in FP64) against the FP64 oracle, through the C ABI.

Tolerances (mixed precision): spectra and two-site tensors 1e-6 absolute (each spectrum has
unit 2-norm; tensors relative to their largest entry), peak probability 1e-6 absolute.
The bound: 3xTF32 keeps about 21 bits of every product and sums in FP32, so the merged
bond matrix carries a relative error of a few 1e-7; singular values move by at most the
2-norm of that error.  Singular values the FP64 path resolves at 1e-16 become noise at the
1e-7 level here, so the cutoff of these cases is 1e-5: every kept value sits well above the
mixed noise floor and every dropped one well below the cutoff (a guard band of 1e-3
relative around eps * s_0 is asserted empty), and the discrete results (bond dimensions,
unswap logs, peaks) must then be identical to the oracle's."""
import numpy as np
import pytest

from oracle import mpo
from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6
EPS_MIXED = 1e-5


def random_state(chi, seed):
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


def two_site(Bj, Bj1):
    return np.einsum("lpm,mqr->lpqr", Bj, Bj1)


def check_mixed_update(chi, bonds, seed, chi_max=256, eps=EPS_MIXED):
    B, lam = random_state(chi, seed)
    n = len(B)
    rng = np.random.default_rng(seed + 100)
    ops = [W.haar_unitary(rng, 16) for _ in bonds]
    ctx = binding.Context(eps=eps, chi_max=chi_max, precision=binding.PRECISION_TF32X3)
    c = ctx.load_gates(n, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    c.set_state(B, lam)
    got_chi = c.apply_updates(bonds, np.array(ops))
    cfg = mpo.Config(eps=eps, chi_max=chi_max)
    st = mpo.MPOState(n)
    st.B = [b.copy() for b in B]
    st.lam = [l.copy() for l in lam]
    for k, j in enumerate(bonds):
        t = st.trial(j, ops[k], cfg)
        thr = cfg.eps * t.s[0]
        assert not (np.abs(t.s - thr) <= 1e-3 * thr).any(), "seed puts a singular value inside the guard band"
        st.commit(j, t)
        assert got_chi[k] == t.count
        np.testing.assert_allclose(c.spectrum(j), st.lam[j], atol=TOL_MIXED, rtol=0)
        ref = two_site(st.B[j], st.B[j + 1])
        got = two_site(c.site(j), c.site(j + 1))
        assert np.max(np.abs(got - ref)) <= TOL_MIXED * max(1.0, np.max(np.abs(ref)))
    c.close()
    ctx.close()


def test_mixed_single_update_ragged_tiles():
    # a 148 x 116 bond matrix: two 128-row tensor-core tiles (one ragged), K = 2 * 50 real
    check_mixed_update([1, 4, 13, 37, 50, 29, 11, 4, 1], [3], seed=1)


def test_mixed_batched_uneven_sizes_and_chi_one():
    check_mixed_update([1, 4, 13, 37, 50, 29, 11, 4, 1], [0, 2, 4, 6], seed=2)
    check_mixed_update([1, 1, 1, 1, 1], [0, 2], seed=4, chi_max=64)


def test_mixed_full_size_chi256():
    """chi_l = chi_m = chi_r = 256: 1024 x 1024 bond matrices, 8 x 4 output tiles, K = 512
    real (16 pipeline stages), two tasks in one launch."""
    check_mixed_update([1, 4, 256, 256, 256, 256, 256, 4, 1], [2, 4], seed=11)


def test_mixed_matches_fp64_path_on_the_same_update():
    """The mixed and the FP64 library paths on one update agree to the mixed tolerance and
    return the same count."""
    chi = [1, 4, 16, 64, 96, 64, 16, 4, 1]
    B, lam = random_state(chi, 21)
    op = W.haar_unitary(np.random.default_rng(5), 16)
    out = {}
    for prec in (binding.PRECISION_FP64, binding.PRECISION_TF32X3):
        ctx = binding.Context(eps=EPS_MIXED, chi_max=256, precision=prec)
        c = ctx.load_gates(len(B), np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
        c.set_state(B, lam)
        cnt = c.apply_updates([3], op[None])
        out[prec] = (cnt[0], c.spectrum(3), two_site(c.site(3), c.site(4)))
        c.close()
        ctx.close()
    a, b = out[binding.PRECISION_FP64], out[binding.PRECISION_TF32X3]
    assert a[0] == b[0]
    assert np.max(np.abs(a[1] - b[1])) <= TOL_MIXED
    assert np.max(np.abs(a[2] - b[2])) <= TOL_MIXED * np.max(np.abs(a[2]))
    # and the mixed result is not bit-identical: the tensor-core path really ran
    assert np.max(np.abs(a[2] - b[2])) > 0.0


@pytest.mark.parametrize("n,seed", [(8, 1), (9, 2)])
def test_mixed_hidden_permutation_end_to_end(n, seed):
    """Hidden permutation + perturbation 0.02: identical plans, unswap logs, layouts, bond
    dimensions and peak as the FP64 oracle at the same cutoff; p_peak within 1e-6."""
    circ = W.hidden_permutation_mirror(n, 20, 0.02, seed=seed)
    kw = dict(eps=EPS_MIXED, chi_max=64, tau=600)
    ref = mpo.contract(circ, mpo.Config(**kw))
    ctx = binding.Context(precision=binding.PRECISION_TF32X3, **kw)
    c = ctx.load_circuit(circ)
    c.contract()
    plan_ref = np.array([[r.side, r.bond, r.kind, r.gate, r.chi] for r in ref.plan], np.int32).reshape(-1, 5)
    assert np.array_equal(c.plan(), plan_ref)
    assert np.array_equal(c.unswap_log(), np.array(ref.unswap_log, np.int32).reshape(-1, 4))
    assert list(c.bond_dims()) == ref.state.bond_dims()
    for b in range(n - 1):
        np.testing.assert_allclose(c.spectrum(b), ref.state.lam[b], atol=TOL_MIXED, rtol=0)
    bits_ref, p_ref, _, _ = mpo.extract_peak(mpo.project_zero(ref))
    bits, p, _ = c.extract_peak()
    assert np.array_equal(bits, bits_ref) and np.array_equal(bits, circ.planted)
    assert abs(p - p_ref) <= TOL_MIXED
    c.close()
    ctx.close()
