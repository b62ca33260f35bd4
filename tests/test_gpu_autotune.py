"""The FP64 Jacobi autotuner (pc_autotune / pc_load_tuning): it times the group widths on the
device, installs the fastest per launch shape and writes a table that loads back; updates run
with the tuned table agree with the oracle as before (the width changes the rounding order
only).  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from paper_2604_21908_gb300 import binding

from test_gpu_parity import check_update

pytestmark = pytest.mark.gpu


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
