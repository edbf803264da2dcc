"""Failure detection on the GPU without a GPU fault.

Each failure is made on the host, and the kernels' own checks must turn it into
the documented status at the next error check, with the CUDA context still
usable afterwards:

* a non-finite population (NaN) at a fluid node -> LBRMT_ERR_NUMERIC (the
  moments' finiteness test of the lattice Boltzmann kernel);
* a population that the step's collision drives beyond the FP16 storage range
  -> LBRMT_ERR_OVERFLOW (the 16-bit store check);
* two solids' bands on one registry tile with one slot per tile ->
  LBRMT_ERR_OVERFLOW (the registry's slot check; the force kernel reads no more
  than the slots);
* a bounded device wait on a barrier that nothing completes ->
  LBRMT_ERR_TIMEOUT (lbrmt_check_bounded_wait).

The injected nodes lie far from every solid's band and only one step runs, so
the bad values never reach the reference-map kernel's index arithmetic.
"""
import time

import numpy as np
import pytest

import scenarios

pytestmark = pytest.mark.gpu

ERR_NUMERIC, ERR_OVERFLOW, ERR_TIMEOUT = -3, -4, -6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12696_gb300 import build
    build.build()


def _one_disk_box():
    # 128^2 periodic box, one disk of radius 8 at (32, 32): the node (100, 100)
    # is more than 80 nodes from its surface, far outside its 11-layer band
    sc = scenarios._base(128, 128, 0, 0, 0.6, name="one_disk_box")
    sc["solids"].append({"x": 32.0, "y": 32.0, "r": 8.0, "rho_s": 1.2, "G": 0.01})
    return sc


def _still_usable():
    import paper_2402_12696_gb300 as pkg
    sim = pkg.Simulation(_one_disk_box(), precision="fp32")
    sim.step(6)
    sim.sync()
    assert np.isfinite(sim.total_mass())
    sim.close()


def test_nan_population_raises_numeric():
    import paper_2402_12696_gb300 as pkg
    sim = pkg.Simulation(_one_disk_box(), precision="fp32")
    sim.step(4)
    f = sim.populations_host()
    f[1, 100, 100] = np.nan
    sim.set_populations_host(f)
    sim.step(1)
    with pytest.raises(pkg.LbrmtError) as ei:
        sim.sync()
    assert ei.value.status == ERR_NUMERIC and "non-finite" in str(ei.value)
    # a pending device error is reported by the wait check instead of running it
    assert pkg.load().lbrmt_check_bounded_wait(sim.h) == ERR_NUMERIC
    sim.close()
    _still_usable()


def test_fp16_store_range_raises_overflow():
    # FP16 storage scales each population plane by a power of two chosen from a
    # bound of its values (|u| <= 0.3, the density differences): for this box,
    # deviations of plane 1 up to 60000 / 2^16 = 0.92 fit.  An upload that puts
    # 1.2 there exceeds the format and raises the overflow flag; one that puts
    # 0.5 does not.
    import paper_2402_12696_gb300 as pkg
    sim = pkg.Simulation(_one_disk_box(), precision="fp16")
    sim.step(4)
    f = sim.populations_host()
    g = f.copy()
    g[1, 100, 100] += 0.5
    sim.set_populations_host(g)
    sim.sync()
    f[1, 100, 100] += 1.2
    with pytest.raises(pkg.LbrmtError) as ei:  # the upload waits for the stream and reports the flag
        sim.set_populations_host(f)
    assert ei.value.status == ERR_OVERFLOW and "16-bit" in str(ei.value)
    sim.close()
    _still_usable()


def test_registry_slot_overflow():
    import paper_2402_12696_gb300 as pkg
    sc = scenarios.contact_pair(gap=0.8, nx=96, ny=64)  # bands overlap on many tiles
    sim = pkg.Simulation(sc, precision="fp32", max_solids_per_tile=1)
    with pytest.raises(pkg.LbrmtError) as ei:  # the initialisation already registers the bands
        sim.step(2)
        sim.sync()
    assert ei.value.status == ERR_OVERFLOW and "max_solids_per_tile" in str(ei.value)
    sim.close()
    ok = pkg.Simulation(sc, precision="fp32", max_solids_per_tile=2)
    ok.step(2)
    ok.sync()
    ok.close()


def test_bounded_wait_gives_up_with_timeout():
    import paper_2402_12696_gb300 as pkg
    sim = pkg.Simulation(_one_disk_box(), precision="fp32")
    sim.step(2)
    sim.sync()
    t0 = time.perf_counter()
    st = pkg.load().lbrmt_check_bounded_wait(sim.h)
    dt = time.perf_counter() - t0
    assert st == ERR_TIMEOUT, st
    assert 0.2 < dt < 60.0, dt  # ~2^31 SM clock cycles
    # the flags are clear again and the simulation steps on
    sim.step(4)
    sim.sync()
    assert sim.steps_done == 6
    sim.close()
