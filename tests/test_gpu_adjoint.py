"""Adjoint of the LBRMT step on the GPU (lbrmt_forward_checkpointed /
lbrmt_backward / LBRMTFunction).

The loss is a function of the solids' final centroids c_s = sum lambda x /
sum lambda (lambda = 1 - H_eps(phi)); the gradients are checked against
central differences, which the discrete adjoint must reproduce to the
differencing error (the branch decisions of the forward run do not change
under the small perturbations):
  * on the GPU in FP64: dL/dG, dL/d(rho_s/rho_f), dL/df body field (a
    direction and single components), with segments of uneven length;
  * against the FP64 oracle (the FP64 reference gradient): dL/dG and
    dL/d(rho_s/rho_f), and dL/df_q(t=0) at single populations;
  * the checkpoint interval does not change the gradients;
  * FP32 gradients agree with FP64 ones to the accuracy of FP32 storage;
  * the autograd function reproduces the C ABI's gradients.
"""
import numpy as np
import pytest

import oracle
import scenarios

pytestmark = pytest.mark.gpu

N, R, G0, RATIO0, T, K = 48, 8.0, 0.02, 1.3, 20, 6
W = np.array([[0.7, -0.4]])  # dL/dc for L = w . c


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12696_gb300 import build
    build.build()
    oracle.build()


def _scenario(body=None):
    if body is None:
        body = scenarios.smooth_body_field(1, N, amp=2e-5)
    return scenarios.adjoint_ldc(N, r=R, G=G0, rho_ratio=RATIO0, body=body)


def _heaviside(phi, eps):
    return np.where(phi <= -eps, 0.0, np.where(phi >= eps, 1.0,
                                                0.5 * (1 + phi / eps + np.sin(np.pi * phi / eps) / np.pi)))


def oracle_centroid(o, sc, s=0):
    phi = o.field("phi", s)
    ny, nx = phi.shape
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    m = np.isfinite(phi) & (phi < sc["eps"])
    lam = 1 - _heaviside(phi[m], sc["eps"])
    return np.array([(lam * X[m]).sum() / lam.sum(), (lam * Y[m]).sum() / lam.sum()])


def _gpu_loss(sim, body, G=G0, ratio=RATIO0, steps=T):
    sim.set_solid_params(0, ratio * sim.sc["rho_f"], G)
    sim.set_body_force_field(body)
    return float((W * sim.forward_checkpointed(steps, K)).sum())


def _close(a, b, rtol, scale=None):
    s = max(abs(b), scale or 0.0)
    return abs(a - b) <= rtol * s


def test_adjoint_matches_central_differences_fp64():
    import paper_2402_12696_gb300 as pkg
    sc = _scenario()
    body = sc["body_field"]
    sim = pkg.Simulation(sc, precision="fp64")
    sim.forward_checkpointed(T, K)
    dG, dr, db = sim.backward(W, body=True)
    db = db.cpu().numpy()
    h = 1e-4 * G0
    fd = (_gpu_loss(sim, body, G=G0 + h) - _gpu_loss(sim, body, G=G0 - h)) / (2 * h)
    assert _close(dG[0], fd, 1e-4), (dG[0], fd)
    h = 1e-4 * RATIO0
    fd = (_gpu_loss(sim, body, ratio=RATIO0 + h) - _gpu_loss(sim, body, ratio=RATIO0 - h)) / (2 * h)
    assert _close(dr[0], fd, 1e-4), (dr[0], fd)
    v = scenarios.smooth_body_field(7, N, amp=1.0)
    fd = (_gpu_loss(sim, body + 1e-6 * v) - _gpu_loss(sim, body - 1e-6 * v)) / 2e-6
    assert _close(float((db * v).sum()), fd, 1e-5), ((db * v).sum(), fd)
    scale = np.abs(db).max()
    for (c, y, x) in [(0, 24, 20), (1, 30, 29), (0, 14, 29), (1, 24, 38)]:
        e = np.zeros_like(body)
        e[c, y, x] = 1.0
        fd = (_gpu_loss(sim, body + 1e-5 * e) - _gpu_loss(sim, body - 1e-5 * e)) / 2e-5
        assert _close(db[c, y, x], fd, 1e-5, scale), (c, y, x, db[c, y, x], fd)
    sim.close()


def test_adjoint_matches_oracle_reference_gradient():
    # FP64 reference gradient: central differences of the FP64 oracle
    import paper_2402_12696_gb300 as pkg
    sc = _scenario()
    sim = pkg.Simulation(sc, precision="fp64")
    sim.forward_checkpointed(T, K)
    dG, dr, _ = sim.backward(W)

    def oloss(G=G0, ratio=RATIO0):
        s2 = dict(sc)
        s2["solids"] = [dict(sc["solids"][0], G=G, rho_s=ratio * sc["rho_f"])]
        o = oracle.Oracle(s2)
        o.step(T)
        val = float((W[0] * oracle_centroid(o, s2)).sum())
        o.close()
        return val

    h = 1e-4 * G0
    assert _close(dG[0], (oloss(G=G0 + h) - oloss(G=G0 - h)) / (2 * h), 1e-4)
    h = 1e-4 * RATIO0
    assert _close(dr[0], (oloss(ratio=RATIO0 + h) - oloss(ratio=RATIO0 - h)) / (2 * h), 1e-4)
    # initial populations, short horizon: dL/df_q(x, 0) at single populations
    steps = 6
    sim.forward_checkpointed(steps, 4)
    _, _, _, d0 = sim.backward(W, f0=True)
    d0 = d0.cpu().numpy()
    base = oracle.Oracle(sc)
    f0 = base.populations()
    base.close()
    scale = np.abs(d0).max()
    for (q, y, x) in [(1, 24, 22), (2, 24, 22), (0, 24, 22), (1, 24, 20), (3, 30, 30), (2, 18, 26)]:
        vals = []
        for sgn in (1, -1):
            o = oracle.Oracle(sc)
            f = f0.copy()
            f[q, y, x] += sgn * 1e-7
            o.set_populations(f)
            o.step(steps)
            vals.append(float((W[0] * oracle_centroid(o, sc)).sum()))
            o.close()
        assert _close(d0[q, y, x], (vals[0] - vals[1]) / 2e-7, 1e-4, scale), (q, y, x)
    sim.close()


def test_checkpoint_interval_does_not_change_gradients():
    import paper_2402_12696_gb300 as pkg
    sc = _scenario()
    sim = pkg.Simulation(sc, precision="fp64")
    out = []
    for k in (1, 7, T):
        sim.forward_checkpointed(T, k)
        dG, dr, db = sim.backward(W, body=True)
        out.append((dG[0], dr[0], db.cpu().numpy()))
    for o in out[1:]:
        assert _close(o[0], out[0][0], 1e-10)
        assert _close(o[1], out[0][1], 1e-10)
        assert np.abs(o[2] - out[0][2]).max() <= 1e-10 * np.abs(out[0][2]).max()
    sim.close()


def test_fp32_gradients_agree_with_fp64():
    import paper_2402_12696_gb300 as pkg
    sc = _scenario()
    res = {}
    for prec in ("fp64", "fp32"):
        sim = pkg.Simulation(sc, precision=prec)
        sim.forward_checkpointed(T, K)
        dG, dr, db = sim.backward(W, body=True)
        res[prec] = (dG[0], dr[0], db.cpu().numpy())
        sim.close()
    a, b = res["fp32"], res["fp64"]
    assert _close(a[0], b[0], 1e-3), (a[0], b[0])
    assert _close(a[1], b[1], 1e-2), (a[1], b[1])
    assert np.abs(a[2] - b[2]).max() <= 1e-3 * np.abs(b[2]).max()


def test_autograd_function_matches_backward():
    import torch
    import paper_2402_12696_gb300 as pkg
    sc = _scenario()
    sim = pkg.Simulation(sc, precision="fp64")
    G = torch.tensor([G0], dtype=torch.float64, requires_grad=True)
    ratio = torch.tensor([RATIO0], dtype=torch.float64, requires_grad=True)
    body = torch.tensor(sc["body_field"], device="cuda", requires_grad=True)
    c = pkg.LBRMTFunction.apply(G, ratio, body, sim, T, K)
    target = c.detach() + torch.tensor([[1.0, -1.0]], dtype=torch.float64)
    loss = ((c - target) ** 2).sum()
    loss.backward()
    dG, dr, db = sim.backward(2 * (c.detach() - target).numpy(), body=True)
    # two reverse sweeps sum their atomic contributions in different orders
    assert _close(G.grad.item(), dG[0], 1e-9)
    assert _close(ratio.grad.item(), dr[0], 1e-9)
    assert torch.allclose(body.grad, db, rtol=0, atol=1e-9 * db.abs().max().item())
    sim.close()


def test_forward_checkpointed_equals_plain_run():
    import paper_2402_12696_gb300 as pkg
    sc = _scenario()
    sim = pkg.Simulation(sc, precision="fp32")
    c = sim.forward_checkpointed(T, K)
    sim2 = pkg.Simulation(sc, precision="fp32")
    sim2.step(T)
    st = sim2.solid_stats()
    assert c[0, 0] == st[0, 1] and c[0, 1] == st[0, 2]
    sim.close()
    sim2.close()


def test_backward_needs_a_forward_run():
    import paper_2402_12696_gb300 as pkg
    sim = pkg.Simulation(_scenario(), precision="fp32")
    with pytest.raises(pkg.LbrmtError, match="ERR_STATE"):
        sim.backward(W)
    sim.close()


@pytest.mark.slow
def _agreements(g, fds, rtol=1e-4):
    """Relative errors of the adjoint gradient g against each central difference."""
    return [abs(g - fd) / abs(fd) for fd in fds]


def test_adjoint_256_cavity_full_length():
    # 256^2 cavity, disk r = 40, 3000 steps, checkpoints every 100: FP64 adjoint
    # against GPU central differences on G and rho_s / rho_f.  Over 3000 steps
    # interface nodes cross phi = 0 (advected <-> extrapolated); a difference
    # whose +-h interval contains such a crossing is not a derivative, and the
    # crossings do not become smaller with h, only rarer.  So four step sizes
    # are taken and the adjoint must match at least two of them: one lucky
    # difference cannot pass the test, and one step size that straddles a
    # crossing cannot fail it.
    import paper_2402_12696_gb300 as pkg
    sc = scenarios.adjoint_ldc(256, r=40.0, G=0.01, rho_ratio=1.0)
    sim = pkg.Simulation(sc, precision="fp64")
    c0 = sim.forward_checkpointed(1, 1)
    target = c0 + np.array([[8.0, -8.0]])
    cT = sim.forward_checkpointed(3000, 100)
    dG, dr, _ = sim.backward(2 * (cT - target))

    def loss(G=0.01, ratio=1.0):
        sim.set_solid_params(0, ratio, G)
        c = sim.forward_checkpointed(3000, 100)
        return float(((c - target) ** 2).sum())

    steps = (1e-5, 1e-6, 1e-7, 3e-8)
    fds = [(loss(G=0.01 + hr * 0.01) - loss(G=0.01 - hr * 0.01)) / (2 * hr * 0.01) for hr in steps]
    errs = _agreements(dG[0], fds)
    assert sum(e < 1e-4 for e in errs) >= 2, (dG[0], fds, errs)
    fds = [(loss(ratio=1.0 + hr) - loss(ratio=1.0 - hr)) / (2 * hr) for hr in steps]
    errs = _agreements(dr[0], fds)
    assert sum(e < 1e-4 for e in errs) >= 2, (dr[0], fds, errs)
    sim.close()


def test_adjoint_256_cavity_body_force_direction():
    # The body-force gradient at the configured size, over a shorter horizon
    # (100 steps, checkpoints every 20): the adjoint's dL/df along two smooth
    # seeded directions against central differences.  Over tens of steps the
    # loss has kinks (interface nodes crossing phi = 0 or the blur-zone edge),
    # so a difference over +-h is the local derivative only when no kink falls
    # inside; measured on this case: at h = 1e-8 the difference matches the
    # adjoint to 3e-8, at h = 1e-5 .. 1e-7 (kinks inside) to 3e-4 .. 4e-4, and
    # at 20 steps every h from 1e-5 down matches.  So the check asks for a
    # match to 1e-6 at one of three tiny step sizes: a kinked difference misses
    # by ~1e-4, and a chance agreement to 1e-6 is not plausible.
    import paper_2402_12696_gb300 as pkg
    body = scenarios.smooth_body_field(3, 256, amp=1e-5)
    sc = scenarios.adjoint_ldc(256, r=40.0, G=0.01, rho_ratio=1.2, body=body)
    sim = pkg.Simulation(sc, precision="fp64")
    c0 = sim.forward_checkpointed(1, 1)
    target = c0 + np.array([[2.0, -1.0]])
    sim.set_body_force_field(body)
    cT = sim.forward_checkpointed(100, 20)
    _, _, db = sim.backward(2 * (cT - target), body=True)
    db = db.cpu().numpy()

    def loss(b):
        sim.set_body_force_field(b)
        c = sim.forward_checkpointed(100, 20)
        return float(((c - target) ** 2).sum())

    for seed in (11, 12):
        v = scenarios.smooth_body_field(seed, 256, amp=1.0)
        g = float((db * v).sum())
        fds = [(loss(body + h * v) - loss(body - h * v)) / (2 * h) for h in (1e-8, 3e-9, 1e-9)]
        errs = _agreements(g, fds)
        assert min(errs) < 1e-6, (seed, g, fds, errs)
    sim.close()
