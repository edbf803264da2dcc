"""The FP32 quantity that sets the density floor of the FP32 parity bound.

The FP32 path stores each population as its deviation g_q = f_q - w_q rho_f
(Sec. 2.3's rest state subtracted).  Where a wall moves, the halfway
bounce-back of Sec. 3.5 puts deviations of 6 w_q rho lid_u into the stored
populations (8e-3 for a lid of 0.05), and one FP32 rounding of a deviation of
that size is ~5e-10.  One step into the 64^2 cavity with a body-force field,
the density deviation is only 8e-5, so rounding the oracle's own exact
populations to FP32 deviations already moves rho by a relative ~1e-5 of it.
Density deviations below 1e-4 rho_f are therefore compared against the floor
1e-4 rho_f (parity_util.FLOORS), where that rounding is a relative 1e-5.
"""
import numpy as np

import oracle
import scenarios
from parity_util import FLOORS

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]


def test_density_floor_is_the_fp32_resolution_of_the_populations():
    sc = scenarios.adjoint_ldc(64, r=12, body=scenarios.smooth_body_field(0, 64, amp=1e-4))
    ref = oracle.Oracle(sc)
    ref.step(1)
    g = ref.populations() - W * sc["rho_f"]     # the stored form (Delta rho = 0: rho_s = rho_f)
    drho = ref.field("rho") - sc["rho_f"]
    rep = np.abs(g.astype(np.float32).astype(np.float64).sum(0) - g.sum(0)).max()
    dmax = np.abs(drho).max()
    ref.close()
    # the largest stored deviation is the lid's bounce-back term
    assert np.abs(g).max() > 6 * W[5, 0, 0] * sc["lid_u"] * 0.9
    # FP32 storage of the exact populations alone: a relative ~1e-5 of the density deviation
    assert rep > 5e-6 * dmax
    # and within 1e-5 of the floor
    assert dmax < FLOORS["rho"] * sc["rho_f"] and rep < 1e-5 * FLOORS["rho"] * sc["rho_f"]
