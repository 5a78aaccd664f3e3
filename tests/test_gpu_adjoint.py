"""The CUDA adjoint (ns_adjoint) against the oracle's adjoint, central finite
differences, and itself under different checkpoint intervals."""
import numpy as np
import pytest
import torch

import oracle
from paper_1705_06149_gb300 import Grid, inputs
from paper_1705_06149_gb300.autograd import kinetic_energy

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _start(dims, moving, seed=12):
    og = oracle.Grid(*dims, re=40.0, u_lid=1.0, rtol=1e-13)
    if not moving:
        return og.zeros()
    rs = inputs.random_state(*dims, seed=seed, sigma=0.3)
    u, v, w, _ = og.project(*rs[:3], rtol=1e-14)
    return [u, v, w, np.zeros(og.shape(3))]


@pytest.mark.parametrize("moving", [False, True])
def test_adjoint_matches_oracle(moving):
    dims, dt, steps = (12, 10, 8), 2e-3, 8
    st0 = _start(dims, moving)
    og = oracle.Grid(*dims, re=40.0, u_lid=1.0, rtol=1e-13)
    Jr, gr, dlr = og.adjoint(st0, dt, steps, rtol=1e-13)
    g = Grid(*dims, re=40.0, u_lid=1.0, poisson_rtol=1e-13, batch=2)
    st = g.state_from([np.stack([a, a]) for a in st0])
    J, grad, dl = g.adjoint(st, dt, steps, ckpt_every=3)
    for b in range(2):
        assert abs(J[b] - Jr) <= 1e-10 * Jr
        assert abs(dl[b] - dlr) <= 1e-9 * abs(dlr)
        vg = np.concatenate([t[b].cpu().numpy().ravel() for t in (grad.u, grad.v, grad.w)])
        vr = np.concatenate([a.ravel() for a in gr])
        # Starting from rest, most faces carry velocities near zero for the
        # first steps, where a rounding-level difference between the two
        # forward runs can change which SMART branch a face takes (and so
        # which piece of the piecewise-linear Jacobian each adjoint uses).
        tol = 1e-9 if moving else 1e-7
        assert rel(vg, vr) <= tol, rel(vg, vr)


def test_fp32_refine_adjoint_matches_oracle():
    """FP32 storage with FP64-accurate refinement: the forward steps, the
    adjoint projections and the adjoint stencils in FP32, against the oracle's
    FP64 adjoint of the same steps (from the start state rounded to FP32)."""
    dims, dt, steps = (12, 10, 8), 2e-3, 8
    st0 = _start(dims, True)
    st0 = [np.asarray(a, dtype=np.float32).astype(np.float64) if c < 3 else a
           for c, a in enumerate(st0)]
    og = oracle.Grid(*dims, re=40.0, u_lid=1.0, rtol=1e-13)
    Jr, gr, dlr = og.adjoint(st0, dt, steps, rtol=1e-13)
    g = Grid(*dims, re=40.0, u_lid=1.0, precision="fp32_refine", batch=2)
    st = g.state_from([np.stack([a, a]) for a in st0])
    J, grad, dl = g.adjoint(st, dt, steps, ckpt_every=3)
    assert grad.u.dtype == torch.float32
    vr = np.concatenate([a.ravel() for a in gr])
    for b in range(2):
        vg = np.concatenate([t[b].double().cpu().numpy().ravel() for t in (grad.u, grad.v, grad.w)])
        e = rel(vg, vr)
        print(f"\nFP32+refine adjoint vs oracle: gradient {e:.2e}, J {abs(J[b] - Jr) / Jr:.2e}, "
              f"dJ/du_lid {abs(dl[b] - dlr) / abs(dlr):.2e}")
        assert e <= 1e-5, e
        assert abs(J[b] - Jr) <= 1e-6 * Jr
        assert abs(dl[b] - dlr) <= 1e-5 * abs(dlr)


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_adjoint_is_deterministic(prec):
    """Every sum of the adjoint has a fixed order (gathered (dR/du)^T mu,
    per-CTA partials of J and dJ/du_lid): two calls give the same bits."""
    dims, dt, steps = (16, 12, 10), 2e-3, 6
    g = Grid(*dims, re=40.0, precision=prec, batch=2)
    st = g.state_from([np.stack([a, a]) for a in _start(dims, True, seed=4)])
    J1, g1, d1 = g.adjoint(st, dt, steps, ckpt_every=2)
    J2, g2, d2 = g.adjoint(st, dt, steps, ckpt_every=2)
    assert J1 == J2 and d1 == d2
    for a, b in zip(g1.fields()[:3], g2.fields()[:3]):
        assert torch.equal(a, b)


def test_checkpoint_interval_does_not_change_the_gradient():
    dims, dt, steps = (10, 10, 10), 2e-3, 7
    st0 = _start(dims, True, seed=3)
    g = Grid(*dims, re=40.0, batch=1)
    st = g.state_from(st0)
    outs = [g.adjoint(st, dt, steps, ckpt_every=c) for c in (1, 3, 7, 100)]
    J0, g0, d0 = outs[0]
    v0 = torch.cat([g0.u.flatten(), g0.v.flatten(), g0.w.flatten()])
    for J, gr, d in outs[1:]:
        # the recomputed states are bit-identical and every sum has a fixed
        # order: the gradient does not depend on the interval at all
        assert J[0] == J0[0]
        v = torch.cat([gr.u.flatten(), gr.v.flatten(), gr.w.flatten()])
        assert torch.equal(v, v0)
        assert d[0] == d0[0]


def test_gradient_matches_central_differences_on_the_gpu():
    dims, dt, steps = (16, 16, 16), 1e-3, 10
    g = Grid(*dims, re=100.0, u_lid=1.0, poisson_rtol=1e-14, batch=1)
    st0 = g.state_from(_start(dims, True, seed=21))
    J, grad, dl = g.adjoint(st0, dt, steps, ckpt_every=4)
    rng = np.random.default_rng(0)

    def objective(state, lid=1.0):
        g.set_lid_speed(lid)
        s = state.clone()
        g.step_fine(s, dt, steps)
        g.set_lid_speed(1.0)
        og = oracle.Grid(*dims)
        return og.kinetic_objective([a[0] for a in s.numpy()])

    h = 1e-6
    for trial in range(4):
        d = [rng.normal(size=tuple(t.shape)) for t in (st0.u, st0.v, st0.w)]
        for c, a in enumerate(d):  # zero on wall-normal faces
            ax = a.ndim - 1 - c
            sl0 = [slice(None)] * a.ndim
            sl1 = [slice(None)] * a.ndim
            sl0[ax] = 0
            sl1[ax] = -1
            a[tuple(sl0)] = 0
            a[tuple(sl1)] = 0
        nrm = np.sqrt(sum(np.sum(a * a) for a in d))
        d = [torch.tensor(a / nrm, device="cuda") for a in d]
        plus = st0.clone()
        minus = st0.clone()
        for c, t in enumerate((plus.u, plus.v, plus.w)):
            t += h * d[c]
        for c, t in enumerate((minus.u, minus.v, minus.w)):
            t -= h * d[c]
        fd = (objective(plus) - objective(minus)) / (2 * h)
        ad = float(sum((gr * dd).sum() for gr, dd in zip((grad.u, grad.v, grad.w), d)))
        assert abs(fd - ad) <= 1e-4 * abs(ad) + 1e-12, (trial, fd, ad)
    fd = (objective(st0, 1.0 + h) - objective(st0, 1.0 - h)) / (2 * h)
    assert abs(fd - dl[0]) <= 1e-4 * abs(dl[0]), (fd, dl[0])


def test_autograd_function_gives_the_adjoint_gradient():
    dims, dt, steps = (10, 10, 10), 2e-3, 5
    g = Grid(*dims, re=40.0, batch=1)
    st0 = g.state_from(_start(dims, True, seed=5))
    u = st0.u.clone().requires_grad_(True)
    v = st0.v.clone().requires_grad_(True)
    w = st0.w.clone().requires_grad_(True)
    lid = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = kinetic_energy(u, v, w, lid, g, dt, steps, 2)
    (2.0 * J.sum()).backward()
    Jr, gr, dl = g.adjoint(st0, dt, steps, 2)
    assert torch.allclose(u.grad, 2.0 * gr.u, rtol=1e-12, atol=0)
    assert abs(float(lid.grad) - 2.0 * dl[0]) <= 1e-12 * abs(dl[0])
    # without a gradient to compute, the forward runs the steps and J alone
    with torch.no_grad():
        J2 = kinetic_energy(st0.u, st0.v, st0.w, torch.tensor(1.0, dtype=torch.float64), g, dt,
                            steps, 2)
    assert abs(float(J2[0]) - Jr[0]) <= 1e-10 * Jr[0]


def test_adjoint_full_size_matches_central_differences():
    """The adjoint workload at full size (64^3 cavity, Re 400, 500 steps of
    1e-3, checkpoints every 25 steps, FP64) from a seeded moving start: the
    gradient along 16 seeded random directions of the initial velocity and the
    derivative with respect to the lid speed agree with central differences
    (h = 1e-6) to 1e-4.  The 32 perturbed runs go as one batch.  The
    FP32+refine adjoint of the same workload meets the same differences to
    1e-4 and the FP64 gradient to 1e-4."""
    from paper_1705_06149_gb300 import State
    n, dt, steps, ckpt, h, ndir = 64, 1e-3, 500, 25, 1e-6, 16
    g = Grid(n, n, n, re=400.0, u_lid=1.0, poisson_rtol=1e-14, batch=2 * ndir)
    st0 = g.state_from(inputs.random_state(n, n, n, seed=31, sigma=0.3))
    g.project(st0)
    _, grad, dl = g.adjoint(st0, dt, steps, ckpt_every=ckpt)
    rng = np.random.default_rng(1)
    dirs = []
    for _ in range(ndir):
        d = [rng.normal(size=tuple(t.shape[1:])) for t in (st0.u, st0.v, st0.w)]
        for c, a in enumerate(d):  # zero on wall-normal faces
            sl0 = [slice(None)] * 3
            sl1 = [slice(None)] * 3
            sl0[2 - c] = 0
            sl1[2 - c] = -1
            a[tuple(sl0)] = 0
            a[tuple(sl1)] = 0
        nrm = np.sqrt(sum(np.sum(a * a) for a in d))
        dirs.append([torch.tensor(a / nrm, device="cuda") for a in d])
    vel = []
    for c, t in enumerate((st0.u, st0.v, st0.w)):
        vel.append(torch.stack([t[0] + s * h * d[c] for d in dirs for s in (1.0, -1.0)]))
    p = st0.p.expand((2 * ndir,) + tuple(st0.p.shape[1:])).contiguous()
    batch = State(*[v.contiguous() for v in vel], p)
    g.step_fine(batch, dt, steps)
    og = oracle.Grid(n, n, n)
    fin = batch.numpy()
    fds = []
    for k, d in enumerate(dirs):
        jp = og.kinetic_objective([fin[c][2 * k] for c in range(3)])
        jm = og.kinetic_objective([fin[c][2 * k + 1] for c in range(3)])
        fd = (jp - jm) / (2 * h)
        fds.append(fd)
        ad = float(sum((gr[0] * dd).sum() for gr, dd in zip((grad.u, grad.v, grad.w), d)))
        assert abs(fd - ad) <= 1e-4 * abs(ad) + 1e-12, (k, fd, ad)
    js = []
    for lid in (1.0 + h, 1.0 - h):
        g.set_lid_speed(lid)
        s = st0.clone()
        g.step_fine(s, dt, steps)
        js.append(og.kinetic_objective([a[0] for a in s.numpy()[:3]]))
    g.set_lid_speed(1.0)
    fd_lid = (js[0] - js[1]) / (2 * h)
    assert abs(fd_lid - dl[0]) <= 1e-4 * abs(dl[0]), (fd_lid, dl[0])
    # the FP32+refine adjoint of the same workload: against the same central
    # differences (of the FP64 forward) and against the FP64 gradient
    g32 = Grid(n, n, n, re=400.0, u_lid=1.0, precision="fp32_refine", batch=1)
    st32 = g32.state_from([t.cpu().numpy() for t in st0.fields()])
    _, grad32, dl32 = g32.adjoint(st32, dt, steps, ckpt_every=ckpt)
    v64 = torch.cat([t[0].flatten() for t in (grad.u, grad.v, grad.w)])
    v32 = torch.cat([t[0].double().flatten() for t in (grad32.u, grad32.v, grad32.w)])
    e32 = float((v32 - v64).norm() / v64.norm())
    print(f"\nFP32+refine adjoint at 64^3 x 500 steps: gradient vs FP64 {e32:.2e}, "
          f"dJ/du_lid {abs(dl32[0] - dl[0]) / abs(dl[0]):.2e}")
    assert e32 <= 1e-4, e32
    for k, d in enumerate(dirs):
        ad = float(sum((gr[0].double() * dd).sum() for gr, dd in
                       zip((grad32.u, grad32.v, grad32.w), d)))
        assert abs(fds[k] - ad) <= 1e-4 * abs(ad) + 1e-12, (k, fds[k], ad)
    assert abs(fd_lid - dl32[0]) <= 1e-4 * abs(dl32[0]), (fd_lid, dl32[0])
    g32.close()
    g.close()
