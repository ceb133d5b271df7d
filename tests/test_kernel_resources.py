"""Register and spill reports of the sweep kernels, read from the ptxas
output of the library build (no GPU needed).

The sweeps are latency-bound: their speed depends on how many gathers each
warp keeps in flight, which ptxas decides within the registers a block of
that size allows.  Guarded here: no sweep, level-solve, fused or Krylov
kernel spills to local memory, and the one-row-per-lane sweep's blocks
(including the narrow configuration's 24 warps for FP64 factors) fit the
register file at one block per SM.
"""
import os

import pytest

import paper_2111_09512_gb300 as silu
from paper_2111_09512_gb300 import _build

NO_SPILL_UNITS = ["kernels_sweep.cu", "kernels_staged.cu", "kernels_fused.cu", "kernels_trisolve.cu",
                  "kernels_krylov.cu"]


@pytest.fixture(scope="module")
def reports():
    silu.build()
    if not all(os.path.exists(os.path.join(_build.BUILD, u + ".ptxas.txt")) for u in NO_SPILL_UNITS):
        _build.build(force=True)  # a library built before the reports were kept
    return {u: _build.kernel_resources(u) for u in NO_SPILL_UNITS}


def test_no_hot_kernel_spills(reports):
    for unit, kernels in reports.items():
        assert kernels, unit
        spilling = {k: v for k, v in kernels.items() if v[1] or v[2]}
        assert not spilling, (unit, spilling)


def test_narrow_sweep_instances_exist_without_spills(reports):
    narrow = {k: v for k, v in reports["kernels_staged.cu"].items()
              if "k_sweep_rows" in k and "Li10ELi24ELi360E" in k}
    # FP64 factor with FP64 output, and with FP32 output (the residual of FP32 factors)
    assert len(narrow) == 2, sorted(narrow)
    for name, (regs, st, ld) in narrow.items():
        assert regs <= 80 and st == 0 and ld == 0, (name, regs, st, ld)


def test_sweep_blocks_fit_the_register_file(reports):
    # k_sweep_rows<MT, VI, VO, CH, W, NNZ>: W warps of 32 threads per block, one block per SM
    for name, (regs, _, _) in reports["kernels_staged.cu"].items():
        if "k_sweep_rows" not in name:
            continue
        args = name.split("k_sweep_rowsI", 1)[1]
        warps = int(args.split("ELi")[1])
        assert warps * 32 * regs <= 65536, (name, warps, regs)
