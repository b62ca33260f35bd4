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
