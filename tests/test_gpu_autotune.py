"""The FP64 Jacobi autotuner (pc_autotune / pc_load_tuning): it times the group widths on the
device, installs the fastest per launch shape and writes a table that loads back; updates run
with the tuned table agree with the oracle as before.  The width changes the speed only: the
sweeps sum each inner product in an order fixed by the row length, so the same update gives
bit-identical spectra and site tensors at widths 1, 2 and 4 (rows of 1024 elements: held in
registers at width 4, streamed in a loop at width 1).  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from paper_2604_21908_gb300 import binding
from paper_2604_21908_gb300 import workloads as W

from test_gpu_parity import check_update, random_state

pytestmark = pytest.mark.gpu

TUNE_LEN, TUNE_PAIRS = 14, 16       # the table's buckets (row length, row pairs per round)


def test_autotune_writes_a_table_that_loads_and_keeps_parity(tmp_path):
    path = str(tmp_path / "jacobi_tuning.txt")
    ms = binding.autotune([(64, 4), (256, 2)], path=path)
    assert ms.shape == (2, 3) and np.all(ms > 0)
    lines = [l for l in open(path) if not l.startswith("#")]
    assert len(lines) == 2
    for l in lines:
        bl, bp, g = (int(x) for x in l.split()[:3])
        assert g in (1, 2, 4)
        k = [1, 2, 4].index(g)
        row = [float(x) for x in l.split()[3:6]]
        assert row[k] == min(row)
    binding.load_tuning(path)
    # a 256 x 256 and a ragged update with the tuned widths installed
    check_update(dict(eps=1e-12, chi_max=256), [1, 4, 16, 64, 64, 64, 16, 4, 1], [3], seed=31)
    check_update(dict(eps=1e-12, chi_max=256), [1, 4, 13, 37, 50, 29, 11, 4, 1], [3], seed=1)


def _install_width(tmp_path, g):
    path = tmp_path / f"width_{g}.txt"
    path.write_text("".join(f"{bl} {bp} {g}\n" for bl in range(TUNE_LEN) for bp in range(TUNE_PAIRS)))
    binding.load_tuning(str(path))


def _updates(chi, bonds, seed):
    B, lam = random_state(chi, seed)
    rng = np.random.default_rng(seed + 100)
    ops = np.array([W.haar_unitary(rng, 16) for _ in bonds])
    ctx = binding.Context(eps=1e-12, chi_max=256)
    c = ctx.load_gates(len(B), np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    c.set_state(B, lam)
    out = [np.asarray(c.apply_updates(bonds, ops)).copy()]
    for j in bonds:
        out += [c.spectrum(j), c.site(j), c.site(j + 1)]
    c.close()
    ctx.close()
    return out


def test_group_width_changes_no_bit_of_the_result(tmp_path):
    runs = []
    try:
        for g in (1, 2, 4):
            _install_width(tmp_path, g)
            # a 1024 x 1024 bond matrix (chi = 256 on both sides) and a ragged 148 x 116 one
            runs.append(_updates([1, 4, 16, 64, 256, 256, 256, 64, 16, 4, 1], [4], seed=5) +
                        _updates([1, 4, 13, 37, 50, 29, 11, 4, 1], [3], seed=1))
    finally:
        _install_width(tmp_path, 0)     # back to the built-in choice
    for r in runs[1:]:
        assert len(r) == len(runs[0])
        for x, y in zip(runs[0], r):
            assert np.array_equal(x, y)
