"""The measurement model behind `roofline.achieved`: bench.algorithmic_bytes on a
hand-made three-level hierarchy, every figure worked out by hand below.

Model: one setup pass over a level is P = 4(n+1) + (4 + w) nnz (w = 4 for the
caller's float weights on the fine level, 8 for the FP64 coarse weights); the
fine level takes 5 passes, a coarsened level 4, the coarsest 2.  One sweep or
power-iteration matvec is B = 4(n+1) + (4 + V) nnz + 2 V n (V = 4 in the FP32
form, 8 on tiny levels); the fine level adds one B for the Rayleigh quotient.
Large levels are charged to the grid-wide kernels, small ones to the one-block
kernel."""
import types

import bench


class FakePlan:
    def __init__(self, levels):
        self.levels = levels
        self.num_levels = len(levels)

    def level_info(self, l):
        return self.levels[l]


def lvl(n, nnz, gs, pi):
    return types.SimpleNamespace(n=n, nnz=nnz, gs_sweeps=gs, pi_iters=pi)


def test_algorithmic_bytes_by_hand():
    plan = FakePlan([lvl(1000, 3996, 2, 1),   # large (n > 500): grid-wide kernels
                     lvl(400, 2000, 2, 1),    # small, not tiny: one-block kernel
                     lvl(20, 60, 2, 30)])     # tiny and coarsest: one-block kernel, FP64 vectors
    b = bench.algorithmic_bytes(plan, fp64=False, w_bytes0=4, tail_max_n=500, tail_max_nnz=10000)
    # level 0: P = 4*1001 + 8*3996 = 35,972, five passes
    assert b["grid_setup"] == 5 * 35972
    # level 0: B = 4*1001 + 8*3996 + 8*1000 = 43,972; 2 sweeps + 1 step + the Rayleigh quotient
    assert b["grid_sweeps"] == 3 * 43972
    assert b["grid_solve"] == 4 * 43972
    # level 1: P = 4*401 + 12*2000 = 25,604 (4 passes); B = 4*401 + 8*2000 + 8*400 = 20,804 (3)
    # level 2: P = 4*21 + 12*60 = 804 (2 passes); B = 4*21 + 12*60 + 16*20 = 1,124 (32)
    assert b["cta"] == 4 * 25604 + 3 * 20804 + 2 * 804 + 32 * 1124


def test_algorithmic_bytes_fp64_form():
    plan = FakePlan([lvl(1000, 3996, 2, 1), lvl(20, 60, 0, 5)])
    b = bench.algorithmic_bytes(plan, fp64=True, w_bytes0=8, tail_max_n=500, tail_max_nnz=10000)
    # level 0: P = 4*1001 + 12*3996 = 51,956; B = 4*1001 + 12*3996 + 16*1000 = 67,956
    assert b["grid_setup"] == 5 * 51956
    assert b["grid_solve"] == 4 * 67956
    # level 1 (coarsest, tiny): P = 804 (2 passes); B = 1,124 (5 steps)
    assert b["cta"] == 2 * 804 + 5 * 1124
