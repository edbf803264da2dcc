"""Checkpoint and resume through the C ABI (lbrmt_save / lbrmt_load).

* A run saved at step n, loaded into a fresh simulation of the same scenario
  and stepped on, gives the same fields, solid statistics and total mass, bit
  for bit, as the run that went on from step n: the checkpoint holds the whole
  state that Algorithm 1 carries from one step to the next.  Checked in the
  four precisions, at an odd step (the other half of every ping-pong pair is
  current), with walls, gravity, a lid, a body-force field and the overlapped
  schedule.
* A simulation rewound to its own checkpoint repeats its steps exactly.
* The loading simulation adopts the checkpoint's tile shape and the solids'
  densities and shear moduli.
* Buffers that are not a checkpoint of a matching simulation are refused with
  LBRMT_ERR_ARG and leave the state as it was.
"""
import numpy as np
import pytest

import scenarios

pytestmark = pytest.mark.gpu

ERR_ARG, ERR_STATE = -1, -8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12696_gb300 import build
    build.build()


def _state(sim, nsolids):
    out = [sim.field_host(n) for n in ("rho", "ux", "uy", "Fx", "Fy", "drho")]
    out += [sim.field_host(n, k) for k in range(nsolids) for n in ("xi_x", "xi_y", "phi")]
    out += [sim.solid_stats(), np.array([sim.total_mass(), sim.steps_done], dtype=np.float64)]
    return out


def _same(a, b):
    assert len(a) == len(b)
    for k, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y, equal_nan=True), k


@pytest.mark.parametrize("at", [0, 37])
@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp16", "bf16"])
def test_resume_is_bit_identical(prec, at):
    # at 0: saved right after initialisation, where the next step's moments
    # have no half-force term yet (the density plane's mark travels with it)
    import paper_2402_12696_gb300 as pkg
    sc = scenarios.settling_small(1)  # walls and gravity
    ns = len(sc["solids"])
    a = pkg.Simulation(sc, precision=prec, tile_x=16)
    a.init()
    a.step(at)
    blob = a.save()
    a.step(40)
    ref = _state(a, ns)
    a.close()
    b = pkg.Simulation(sc, precision=prec, tile_x=16)
    b.load(blob)  # initialises b first
    assert b.steps_done == at
    b.step(40)
    _same(ref, _state(b, ns))
    b.close()


@pytest.mark.parametrize("case", ["mixing_small", "ldc_body_field", "ldc_disk"])
def test_rewind_to_own_checkpoint(case):
    import paper_2402_12696_gb300 as pkg
    sc = {"mixing_small": lambda: scenarios.mixing_small(0),
          "ldc_body_field": lambda: scenarios.adjoint_ldc(64, r=12, body=scenarios.smooth_body_field(0, 64, amp=1e-4)),
          "ldc_disk": scenarios.ldc_disk_64}[case]()
    ns = len(sc["solids"])
    sim = pkg.Simulation(sc, precision="fp32", tile_x=16, use_tma=False)  # the overlapped schedule
    sim.step(21)
    blob = sim.save()
    sim.step(30)
    first = _state(sim, ns)
    sim.load(blob)
    assert sim.steps_done == 21
    sim.step(30)
    _same(first, _state(sim, ns))
    sim.close()


def test_load_adopts_tile_shape_and_solid_parameters():
    import paper_2402_12696_gb300 as pkg
    sc = scenarios.settling_small(0)
    ns = len(sc["solids"])
    a = pkg.Simulation(sc, precision="fp32", tile_x=16)
    a.set_solid_params(0, 1.3, 0.03)
    a.step(12)
    blob = a.save()
    a.step(15)
    ref = _state(a, ns)
    b = pkg.Simulation(sc, precision="fp32", tile_x=64)
    b.step(3)
    b.load(blob)
    assert b.tile_x == 16
    b.step(15)
    _same(ref, _state(b, ns))
    # the adopted parameters persist: both return to the same initial state
    a.reset()
    b.reset()
    a.step(10)
    b.step(10)
    _same(_state(a, ns), _state(b, ns))
    a.close()
    b.close()


def test_mismatched_buffers_are_refused():
    import torch
    import paper_2402_12696_gb300 as pkg
    sc = scenarios.settling_small(0)
    ns = len(sc["solids"])
    a = pkg.Simulation(sc, precision="fp32", tile_x=16)
    with pytest.raises(pkg.LbrmtError) as ei:
        a.save()  # not initialised yet
    assert ei.value.status == ERR_STATE
    a.step(8)
    blob = a.save()
    b = pkg.Simulation(sc, precision="fp32", tile_x=16)
    b.step(5)
    before = _state(b, ns)
    others = [pkg.Simulation(scenarios.settling_small(1), precision="fp32", tile_x=16),  # other solids
              pkg.Simulation(sc, precision="fp64", tile_x=16)]                           # other precision
    sc2 = dict(sc)
    sc2["tau"] = sc["tau"] * 0.99
    others.append(pkg.Simulation(sc2, precision="fp32", tile_x=16))                      # other tau
    for o in others:
        with pytest.raises(pkg.LbrmtError) as ei:
            o.load(blob)
        assert ei.value.status == ERR_ARG
        o.close()
    bad = blob.clone()
    bad[0] ^= 0xFF  # not a checkpoint
    for buf in (blob[: blob.numel() // 2], bad, torch.zeros(64, dtype=torch.uint8, device=blob.device)):
        with pytest.raises(pkg.LbrmtError) as ei:
            b.load(buf)
        assert ei.value.status == ERR_ARG
    _same(before, _state(b, ns))
    a.close()
    b.close()
