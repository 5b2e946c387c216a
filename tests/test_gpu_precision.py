"""The precision modes of the solve kernel (mmpc_params.precision) on the
16384-goal, 30-obstacle, N = 200, n = 16 workload at its full size: the
operands of the basis products rounded as the tensor cores take them (TF32,
BF16, each also as hi + lo), FP32 accumulation, 100 iterations.  Every 256th
trajectory is compared with the FP64 oracle (the exact solve); the test prints
the error table and checks what the arithmetic fixes:

* FP32 (mode 0) is the unchanged kernel;
* rounding the operands moves the result away from the exact solve, and the
  hi + lo split brings each dtype back towards it (split error <= plain);
* because the kernel contracts residuals (the increment form of Eq.
  lin_solve_xy_2), the operand errors scale with small quantities: with the
  hi + lo split both TF32 and BF16 keep 90 % of the well-conditioned
  trajectories within 1e-3 m, like FP32, while BF16 alone misses the bar on
  most of them.
"""
import numpy as np
import pytest

import parity_utils as U
from paper_2109_10392_gb300 import mmpc, scenes

pytestmark = pytest.mark.gpu

NAMES = {mmpc.MMPC_PREC_FP32: "fp32", mmpc.MMPC_PREC_TF32: "tf32", mmpc.MMPC_PREC_TF32_SPLIT: "tf32 hi+lo",
         mmpc.MMPC_PREC_BF16: "bf16", mmpc.MMPC_PREC_BF16_SPLIT: "bf16 hi+lo"}


def test_precision_modes_error_table(capsys):
    sc = scenes.scene_custom(31, 16384, 30, N=200, n=16)
    params = dict(sc.params, tol=0.0)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    sel = np.arange(0, len(goals), 256)
    orc = U.oracle_solve(params, ego, obst, goals[sel])
    sens = U.sensitivity(params, ego, obst, goals[sel], orc["coef"], trials=1)
    good = sens < U.SENS_TOL
    rows, med, share = [], {}, {}
    for mode in NAMES:
        gpu = U.gpu_solve(dict(params, precision=mode), ego, obst, goals)
        coef = gpu["coef"][sel]
        assert np.all(np.isfinite(gpu["coef"])), NAMES[mode]
        err = U.pos_err(params, coef, orc["coef"])
        med[mode] = float(np.median(err[good]))
        share[mode] = float(np.mean(err[good] <= U.POS_TOL))
        rows.append(f"  {NAMES[mode]:>10}: parity set ({good.sum()}) median {med[mode]:.2e} max "
                    f"{err[good].max():.2e} m, share <= 1e-3 m {np.mean(err[good] <= U.POS_TOL):.2f}; "
                    f"all sampled median {np.median(err):.2e} m")
    with capsys.disabled():
        print(f"\n[precision modes, N = 200, n = 16, m = 30, sample {len(sel)} of 16384]")
        print("\n".join(rows))
    fp32, tf32, tf32s, bf16, bf16s = (mmpc.MMPC_PREC_FP32, mmpc.MMPC_PREC_TF32, mmpc.MMPC_PREC_TF32_SPLIT,
                                      mmpc.MMPC_PREC_BF16, mmpc.MMPC_PREC_BF16_SPLIT)
    assert med[tf32s] <= med[tf32] and med[bf16s] <= med[bf16]
    assert share[tf32s] >= 0.9 and share[bf16s] >= 0.9 and share[fp32] >= 0.9
    assert med[tf32s] <= 2 * med[fp32] and med[bf16s] <= 2 * med[fp32]
    assert share[bf16] < 0.5 and med[bf16] > 1e-3


def test_precision_mode_arguments():
    """Precision modes exist in the pair kernel with 128 threads and n > 12;
    other shapes are refused at setup, and batches refuse such contexts."""
    base = dict(scenes.scene_custom(1, 4, 3, N=200, n=16).params)
    for bad in (dict(base, precision=2, N=100), dict(base, precision=2, n=12), dict(base, precision=2, variant=1),
                dict(base, precision=5)):
        with pytest.raises(mmpc.MmpcError):
            mmpc.Solver(bad, 3)
    s = mmpc.Solver(dict(base, precision=2), 3)
    sc = scenes.scene_custom(1, 4, 3, N=200, n=16)
    import torch
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0")  # noqa: E731
    with pytest.raises(mmpc.MmpcError):
        mmpc.Batch([dict(params=dict(base, precision=2), ego=t(sc.ego), obst=t(sc.obst), goals=t(sc.goals), solver=s)],
                   sc.meta)
    s.close()
