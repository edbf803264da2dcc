"""lbrmt_total_mass_noalloc: the total mass without any device allocation.

Some callers cannot allocate device memory where they need this diagnostic
(for instance while recording a stream capture that must stay free of
allocation nodes, or after their memory pool has been frozen).  The entry
point keeps its partial sums in a fixed device array inside the library, so
these checks call it through the C ABI and compare it with lbrmt_total_mass,
which reduces partial sums that the library allocated.

lbrmt_total_mass reports the mass of the populations that the last step read,
so each comparison takes the no-allocation sum of the current populations,
advances one step and then reads lbrmt_total_mass: both describe the same
populations and differ only in summation order.  Two rounds run back to back
to show that the shared array's leftover contents do not leak into the next
call.  This file is collected last; it passes on its own in a fresh process
as well as after the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the relative bounds of the total-mass check in test_gpu_parity.py
TOL = {"fp64": 1e-9, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12696_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_total_mass_matches_allocating_entry_point(prec):
    import torch
    import scenarios
    import paper_2402_12696_gb300 as pkg

    sim = pkg.Simulation(scenarios.mixing_small(1), precision=prec)
    sim.init()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=sim.device)
    for _ in range(2):
        sim.step(4)
        sim.sync()
        allocs_before = sim._alloc.n_alloc
        pkg.lbrmt_total_mass_noalloc(sim.h, 0, out.data_ptr())
        sim.sync()
        got = float(out.cpu()[0])
        assert sim._alloc.n_alloc == allocs_before  # the library asked for no memory
        sim.step(1)
        ref = sim.total_mass()
        assert np.isfinite(got)
        assert abs(got - ref) <= TOL[prec] * abs(ref), (prec, got, ref)
        out.fill_(float("nan"))
    sim.close()


def test_noalloc_rejects_an_uninitialised_simulation():
    import torch
    import scenarios
    import paper_2402_12696_gb300 as pkg

    sim = pkg.Simulation(scenarios.mixing_small(0), precision="fp32")
    out = torch.zeros(1, dtype=torch.float64, device=sim.device)
    with pytest.raises(pkg.LbrmtError):
        pkg.lbrmt_total_mass_noalloc(sim.h, 0, out.data_ptr())
    sim.close()
