"""pc_factorise_noalloc, the allocation-free bond factorisation for callers that cannot call
cudaMalloc, checked against the library's regular two-site update (pc_apply_updates) on the
same bond matrices: same count, spectra within TOL_SPEC, and the same kept right singular
subspace (its projector, which does not depend on the phase of each vector) within TOL_AMP.
Two different matrices (a wide one, factorised through its rows, and a tall one, through
its columns) and the first again, in a row, so the shared scratch is reused.  Further shapes
(odd, single row or column, the 256 x 256 limit, cutoff active) against numpy's SVD, and a
check that repeated calls allocate no device memory."""
import numpy as np
import pytest

from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SPEC = 1e-10
TOL_AMP = 1e-10


def state(chi, seed):
    rng = np.random.default_rng(seed)
    B = []
    for j in range(len(chi) - 1):
        cl, cr = chi[j], chi[j + 1]
        z = rng.standard_normal((cl, 4, cr)) + 1j * rng.standard_normal((cl, 4, cr))
        B.append(z / np.linalg.norm(z))
    lam = [W.geometric_spectrum(chi[b + 1], 8.0) for b in range(len(chi) - 2)]
    return B, lam


def bond_matrix(B, lam, j, u16):
    theta0 = np.einsum("lpm,mqr->lpqr", B[j], B[j + 1])
    theta0 = np.einsum("PQpq,lpqr->lPQr", u16.reshape(4, 4, 4, 4), theta0)
    lam_l = lam[j - 1] if j > 0 else np.ones(1)
    return (lam_l[:, None, None, None] * theta0).reshape(4 * B[j].shape[0], 4 * B[j + 1].shape[2])


def test_noalloc_factorisation_matches_regular_update():
    import torch

    chi = [1, 4, 48, 40, 4, 1]        # bond 1: 16 x 160 (rows); bond 2: 192 x 16 (columns)
    eps, chi_max = 1e-12, 64
    B, lam = state(chi, 3)
    rng = np.random.default_rng(4)
    ops = {1: W.haar_unitary(rng, 16), 2: W.haar_unitary(rng, 16)}
    for j in (1, 2, 1):
        ctx = binding.Context(eps=eps, chi_max=chi_max)
        c = ctx.load_gates(len(B), np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
        c.set_state(B, lam)
        ref_count = int(c.apply_updates([j], ops[j][None])[0])
        ref_s = c.spectrum(j)
        ref_vh = c.site(j + 1).reshape(ref_count, -1)
        c.close()
        ctx.close()

        x = bond_matrix(B, lam, j, ops[j])
        m, n = x.shape
        dev = torch.device("cuda")
        xt = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], -1))).to(dev)
        kmax = min(m, n, chi_max)
        s_out = torch.zeros(kmax, dtype=torch.float64, device=dev)
        vh_out = torch.zeros(kmax, n, 2, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        k = binding.factorise_noalloc(xt.data_ptr(), m, n, eps, chi_max, s_out.data_ptr(), vh_out.data_ptr())
        assert k == ref_count
        s = s_out.cpu().numpy()[:k]
        vh = vh_out.cpu().numpy()[:k]
        vh = vh[..., 0] + 1j * vh[..., 1]
        np.testing.assert_allclose(s, ref_s, atol=TOL_SPEC, rtol=0)
        assert np.max(np.abs(vh @ vh.conj().T - np.eye(k))) < TOL_AMP
        proj, proj_ref = vh.conj().T @ vh, ref_vh.conj().T @ ref_vh
        assert np.max(np.abs(proj - proj_ref)) < TOL_AMP


def _factorise(x, eps, chi_max):
    import torch
    m, n = x.shape
    dev = torch.device("cuda")
    xt = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], -1))).to(dev)
    kmax = min(m, n, chi_max)
    s_out = torch.zeros(kmax, dtype=torch.float64, device=dev)
    vh_out = torch.zeros(kmax, n, 2, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    k = binding.factorise_noalloc(xt.data_ptr(), m, n, eps, chi_max, s_out.data_ptr(), vh_out.data_ptr())
    s = s_out.cpu().numpy()[:k]
    vh = vh_out.cpu().numpy()[:k]
    return k, s, vh[..., 0] + 1j * vh[..., 1]


def _matrix(m, n, seed, decay):
    """m x n complex matrix with singular values exp(-decay k), random singular vectors."""
    rng = np.random.default_rng(seed)
    r = min(m, n)
    u, _ = np.linalg.qr(rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r)))
    v, _ = np.linalg.qr(rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))
    s = np.exp(-decay * np.arange(r))
    return (u * s[None, :]) @ v.conj().T


@pytest.mark.parametrize("m,n,decay,chi_max", [
    (7, 33, 0.5, 64),       # odd row count: the Jacobi pads one row
    (33, 7, 0.5, 64),       # tall: factorised through its 7 columns
    (1, 5, 0.0, 8),         # a single row
    (5, 1, 0.0, 8),         # a single column
    (256, 256, 0.2, 64),    # the size limit, widest Jacobi group, cap active
    (200, 120, 0.25, 256),  # cutoff active: exp(-0.25 k) crosses 1e-10 between k = 92 and 93
])
def test_noalloc_shapes_against_numpy_svd(m, n, decay, chi_max):
    """Count, kept spectrum and the kept right singular subspace against numpy's SVD of the
    same matrix under the same rule (keep s_k > eps s_0, at least 1, at most chi_max,
    renormalise to unit 2-norm)."""
    eps = 1e-10
    x = _matrix(m, n, seed=m * 1000 + n, decay=decay)
    _, s_ref, vh_ref = np.linalg.svd(x, full_matrices=False)
    k_ref = max(1, min(int(np.sum(s_ref > eps * s_ref[0])), chi_max))
    k, s, vh = _factorise(x, eps, chi_max)
    assert k == k_ref
    np.testing.assert_allclose(s, s_ref[:k] / np.linalg.norm(s_ref[:k]), atol=TOL_SPEC, rtol=0)
    assert np.max(np.abs(vh @ vh.conj().T - np.eye(k))) < TOL_AMP
    # the rank-k truncation X V V^dagger is well conditioned whatever the spectrum; a vector whose
    # singular value sits near the rounding level of X is not, so the projector itself is
    # compared on the vectors above 1e-6 s_0 only
    x_k, x_k_ref = x @ (vh.conj().T @ vh), x @ (vh_ref[:k].conj().T @ vh_ref[:k])
    assert np.max(np.abs(x_k - x_k_ref)) < 1e-12 * np.max(np.abs(x))
    w = int(np.sum(s_ref[:k] > 1e-6 * s_ref[0]))
    proj, proj_ref = vh[:w].conj().T @ vh[:w], vh_ref[:w].conj().T @ vh_ref[:w]
    assert np.max(np.abs(proj - proj_ref)) < 1e-9


def test_noalloc_allocates_nothing():
    """After a first call (which resolves the scratch array's address and loads the kernels)
    repeated calls change neither the device memory torch has allocated nor the device's
    free memory."""
    import torch
    x = _matrix(96, 80, seed=5, decay=0.1)
    dev = torch.device("cuda")
    xt = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], -1))).to(dev)
    s_out = torch.zeros(64, dtype=torch.float64, device=dev)
    vh_out = torch.zeros(64, 80, 2, dtype=torch.float64, device=dev)
    binding.factorise_noalloc(xt.data_ptr(), 96, 80, 1e-10, 64, s_out.data_ptr(), vh_out.data_ptr())
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        binding.factorise_noalloc(xt.data_ptr(), 96, 80, 1e-10, 64, s_out.data_ptr(), vh_out.data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc1
    assert torch.cuda.mem_get_info()[0] == free1


def test_noalloc_rejects_sizes_beyond_the_limit():
    with pytest.raises(binding.PcError) as e:
        binding.factorise_noalloc(1, 257, 4, 1e-10, 8, 1, 1)
    assert e.value.status == -1
