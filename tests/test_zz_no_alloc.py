"""lbrmt_total_mass_noalloc: the total mass without any device allocation.

Some callers cannot allocate device memory where they need this diagnostic
(a loop running after its memory pool has been frozen, a device whose memory
belongs to another allocator).  The entry point keeps its partial sums in a
fixed device array inside the library, so these checks call it through the C
ABI and compare it with two other routes to the same number:

* lbrmt_total_mass, the allocating entry point, on the same populations;
* the FP64 sum of rho - rho_f over the density field (lbrmt_read_fields).

Before each call known amounts of mass are added to the rest population at a
fluid node and at nodes inside a solid (on a registered tile, where the
stored rest population is relative to the density difference Delta rho), so a
sum that dropped the populations, the rest base or the right step's registry
and force pool would miss them.  Two rounds run back to back, at both step
parities, so the shared array's leftover contents cannot leak into the next
call.  This file is collected last; it passes on its own in a fresh process as
well as after the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# absolute bound, per node: every route sums the same stored values in FP64
# (only the order differs)
TOL = 1e-12


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

    sc = scenarios.mixing_small(1)
    sim = pkg.Simulation(sc, precision=prec)
    sim.init()
    P, rf = sc["nx"] * sc["ny"], sc["rho_f"]
    s0 = sc["solids"][0]
    i0, j0 = int(round(s0["x"])) % sc["nx"], int(round(s0["y"])) % sc["ny"]
    nodes = [(j0, i0), ((j0 + 2) % sc["ny"], i0), (3, 5)]  # two inside solid 0, one in the fluid
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=sim.device)

    def noalloc():
        allocs_before = sim._alloc.n_alloc
        pkg.lbrmt_total_mass_noalloc(sim.h, 0, out.data_ptr())
        sim.sync()
        got = float(out.cpu()[0])
        assert sim._alloc.n_alloc == allocs_before  # the library asked for no memory
        assert np.isfinite(got)
        out.fill_(float("nan"))
        return got

    sim.step(4)
    for rnd in range(2):  # after 4 and after 5 steps: both step parities
        sim.sync()
        m0 = noalloc()
        f = sim.populations_host()
        dm = [2e-3 * (k + 1) * (1 if rnd == 0 else -1) for k in range(len(nodes))]
        for (j, i), d in zip(nodes, dm):
            f[0, j, i] += d
        sim.set_populations_host(f)
        got = noalloc()
        dev = got - rf * P
        assert abs(dev) > 1.0  # the solids' density difference is part of the sum
        # the added mass, and the density field's own FP64 sum
        assert abs((got - m0) - sum(dm)) <= 1e-9 * P, (prec, got - m0, dm)
        field = float((sim.field_host("rho") - rf).sum())
        assert abs(dev - field) <= TOL * P, (prec, dev, field)
        # the allocating entry point on the same populations
        ref = sim.total_mass()
        assert abs(got - ref) <= TOL * P, (prec, got, ref)
        sim.step(1)
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
