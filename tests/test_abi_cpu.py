"""CPU checks of the C-ABI library: it builds and loads, exports every symbol that
include/peaked_mpo.h declares, and its host-only router emits the same absorption plan as
the oracle (Sec. II.A transpilation, Algorithm 1 layer order) record for record."""
import os
import re

import numpy as np
import pytest

from oracle import mpo
from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "peaked_mpo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(binding.EXPORTS) | {"pc_version"}
    assert b"sm_103a" in lib.pc_version()


def oracle_routing_plan(circuit):
    """The oracle's plan with the tensor work switched off (unswapping off, tau infinite)."""
    cfg = mpo.Config(tau=float("inf"), unswap_enabled=False)
    ctr = mpo.Contraction(circuit, cfg)
    ctr.state.apply = lambda j, u16, cfg: 0
    ctr.state.apply_one_site = lambda j, g2, side: None
    res = ctr.run()
    return np.array([[r.side, r.bond, r.kind, r.gate] for r in res.plan], dtype=np.int32).reshape(-1, 4)


@pytest.mark.parametrize("maker", [
    lambda: W.workload_line12(0),
    lambda: W.hidden_permutation_mirror(12, 40, 0.02, seed=3),
    lambda: W.random_circuit(9, 60, seed=2),
    lambda: W.random_circuit(7, 30, seed=5, line=True),
    lambda: W.workload_unswap28(0),
    lambda: W.hqap_like_mirror(56, 918, 27, 0.1, seed=0),     # the paper's shape: 1,917 two-qubit gates
])
def test_router_plan_matches_oracle(maker):
    c = maker()
    ref = oracle_routing_plan(c)
    got = binding.plan_routing(c.n_qubits, c.pairs, c.split_index)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_plan_routing_rejects_bad_pairs():
    with pytest.raises(binding.PcError):
        binding.plan_routing(4, np.array([[0, 0]]), 0)
    with pytest.raises(binding.PcError):
        binding.plan_routing(4, np.array([[0, 4]]), 0)


def test_projected_bytes_matches_its_definition():
    """pc_projected_bytes (host-only): site store at the bond capacities (1 at the ends, chi_max
    inside), spectra, right environments plus one chi_max^2 scratch, the peak-search pool of 4096
    vectors and five buffers per sample (at most 4096 samples at a time), in complex doubles."""
    def expected(n, chi, s):
        cap = [1] + [chi] * (n - 1) + [1]
        sites = sum(cap[j] * 4 * cap[j + 1] for j in range(n)) * 16
        env = sum(cap[j] * cap[j] for j in range(n)) * 16
        return sites + max(1, n - 1) * chi * 8 + env + chi * chi * 16 + 4096 * chi * 16 + min(s, 4096) * chi * 5 * 16

    for n, chi, s in [(2, 1, 0), (8, 64, 0), (28, 256, 1000), (56, 1024, 10000)]:
        assert binding.projected_bytes(n, chi, s) == expected(n, chi, s)
    assert binding.projected_bytes(28, 512, 0) > binding.projected_bytes(28, 256, 0)
    assert binding.load().pc_projected_bytes(1, 64, 0) == -1
    assert binding.load().pc_projected_bytes(8, 0, 0) == -1


def test_config_validation_and_no_gpu_fails_loudly():
    """Out-of-range settings are rejected before any device call; without a GPU, creating a
    context fails with PC_ERR_CUDA (there is no CPU fallback)."""
    import ctypes as C

    import torch

    lib = binding.load()
    h = C.c_void_p()
    for bad in (dict(chi_max=0), dict(chi_max=2048), dict(eps=-1.0), dict(tau=0.0), dict(unswap_mode=3),
                dict(precision=2), dict(side_mode=2), dict(precondition_sweeps=0), dict(jacobi_max_sweeps=0)):
        cfg = binding.default_config(**bad)
        assert lib.pc_create(C.byref(cfg), C.byref(h)) == -1, bad
    if not torch.cuda.is_available():
        cfg = binding.default_config()
        assert lib.pc_create(C.byref(cfg), C.byref(h)) == -7
        with pytest.raises(binding.PcError):
            binding.Server(max_resident=1, memory_budget=1 << 20)


def test_tuning_table_is_parsed_on_the_host(tmp_path):
    """pc_load_tuning (host code, no GPU): '#' lines are comments, widths 1, 2, 4 are installed
    and 0 restores the built-in choice; a file with no valid line or no file is rejected."""
    good = tmp_path / "tuning.txt"
    good.write_text("# len_bucket pairs_bucket width ms(w=1) ms(w=2) ms(w=4)\n"
                    "10 2 4 1.0 2.0 3.0\n10 3 1 1.0 2.0 3.0\n10 2 0\n10 3 0\n")
    binding.load_tuning(str(good))
    bad = tmp_path / "bad.txt"
    bad.write_text("# no entry\n10 2 3\n")
    with pytest.raises(binding.PcError):
        binding.load_tuning(str(bad))
    with pytest.raises(binding.PcError):
        binding.load_tuning(str(tmp_path / "missing.txt"))
