"""GPU adjoint of the mean drag on a fixed sphere against the tangent-linear
oracle (oracle/tangent.cpp) and central differences.

FP64: forces and J within 1e-10 of the oracle, gradients within 1e-9;
checkpoint intervals change nothing (bit for bit).  FP32 at the full
differentiation workload (64^3, d = 12, 500 steps, checkpoints every 50):
within 1e-4 of the FP64 tangent-linear oracle and of FP64 central
differences.  All calls go through the C ABI (and torch.autograd on top).
"""
import numpy as np
import pytest

from paper_2103_10882_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L
    L._native.load()
    return L


SMALL = dict(shape=(24, 24, 24), pos=(12.3, 11.6, 12.2), diameter=6.0, tau=0.7, force=1e-5, steps=30)


def make_sim(lib, shape, pos, diameter, tau, precision):
    s = lib.Simulation(shape, precision=precision, tau=tau)
    s.add_sphere(pos, diameter, 1.0)
    s.set_fixed(True)
    return s


def forward(lib, sim, tau, force, u0, steps, interval, axis=0):
    """(J, per-step forces, device u0) through the C ABI."""
    import torch
    sim.set_tau(tau)
    sim.set_body_force(force)
    dev = torch.device("cuda")
    u = torch.as_tensor(np.ascontiguousarray(u0), dtype=torch.float64, device=dev).contiguous()
    J = torch.empty((), dtype=torch.float64, device=dev)
    forces = torch.empty((steps, 3), dtype=torch.float64, device=dev)
    lib.lbmp_drag_forward(sim.h, u.data_ptr(), steps, interval, axis, J.data_ptr(), forces.data_ptr())
    torch.cuda.synchronize()
    return J.item(), forces.cpu().numpy(), u


def run(lib, sim, tau, force, u0, steps, interval, axis=0):
    """(J, dJ/dtau, dJ/dF[3], dJ/du0) through the C ABI."""
    import torch
    J, _, u = forward(lib, sim, tau, force, u0, steps, interval, axis)
    dev = u.device
    one = torch.ones((), dtype=torch.float64, device=dev)
    gt = torch.empty((), dtype=torch.float64, device=dev)
    gf = torch.empty(3, dtype=torch.float64, device=dev)
    gu = torch.empty_like(u)
    lib.lbmp_drag_backward(sim.h, one.data_ptr(), gt.data_ptr(), gf.data_ptr(), gu.data_ptr())
    torch.cuda.synchronize()
    sim.check()
    return J, gt.item(), gf.cpu().numpy(), gu.cpu().numpy()


def test_fp64_forward_and_gradients_match_tangent_oracle(orc, lib):
    c = SMALL
    u0 = workloads.fourier_velocity_field(c["shape"], 2, 1e-2, 21)
    du = workloads.fourier_velocity_field(c["shape"], 3, 1.0, 22)
    F = (c["force"], 0.0, 0.0)
    sim = make_sim(lib, c["shape"], c["pos"], c["diameter"], c["tau"], "fp64")
    _, fg, _ = forward(lib, sim, c["tau"], F, u0, c["steps"], 7)
    J, gt, gf, gu = run(lib, sim, c["tau"], F, u0, c["steps"], 7)
    args = (c["shape"], c["tau"], c["pos"], c["diameter"], c["steps"])
    Jo, dtau, forces = orc.drag_tangent(*args, u0=u0, body_force=F, dtau=1.0)
    assert J == pytest.approx(Jo, rel=1e-10)
    assert np.abs(fg - forces).max() <= 1e-10 * np.abs(forces).max()
    assert gt == pytest.approx(dtau, rel=1e-9)
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        _, dF, _ = orc.drag_tangent(*args, u0=u0, body_force=F, dforce=e)
        assert gf[a] == pytest.approx(dF, rel=1e-9, abs=1e-9 * abs(gf).max())
    _, dU, _ = orc.drag_tangent(*args, u0=u0, body_force=F, du0=du)
    assert float((gu * du).sum()) == pytest.approx(dU, rel=1e-9)
    # other force components of the objective
    J1, gt1, _, _ = run(lib, sim, c["tau"], F, u0, c["steps"], 7, axis=2)
    Jo1, d1, _ = orc.drag_tangent(*args, u0=u0, body_force=F, dtau=1.0, axis=2)
    assert J1 == pytest.approx(Jo1, rel=1e-10, abs=1e-12 * abs(Jo))
    assert gt1 == pytest.approx(d1, rel=1e-9, abs=1e-9 * abs(dtau))
    sim.close()


def test_checkpoint_interval_changes_nothing(lib):
    c = SMALL
    u0 = workloads.fourier_velocity_field(c["shape"], 2, 1e-2, 21)
    sim = make_sim(lib, c["shape"], c["pos"], c["diameter"], c["tau"], "fp64")
    ref = run(lib, sim, c["tau"], (c["force"], 0, 0), u0, c["steps"], 1)
    for k in (4, 7, 30, 64):
        got = run(lib, sim, c["tau"], (c["force"], 0, 0), u0, c["steps"], k)
        assert got[0] == ref[0] and got[1] == ref[1]
        assert np.array_equal(got[2], ref[2]) and np.array_equal(got[3], ref[3])
    sim.close()


def test_simple_bounce_back_and_rest_state(orc, lib):
    """Simple bounce-back links (delta = 1/2), and the fluid at rest without
    forcing: J = 0 and every gradient equals the oracle's."""
    import torch
    c = SMALL
    sim = lib.Simulation(c["shape"], precision="fp64", tau=0.8, boundary="sbb")
    sim.add_sphere(c["pos"], c["diameter"], 1.0)
    sim.set_fixed(True)
    u0 = np.zeros((3,) + tuple(reversed(c["shape"])))
    J, gt, gf, gu = run(lib, sim, 0.8, (0, 0, 0), u0, 12, 5)
    assert abs(J) < 1e-15
    args = (c["shape"], 0.8, c["pos"], c["diameter"], 12)
    _, dF, _ = orc.drag_tangent(*args, boundary="sbb", dforce=(1, 0, 0))
    assert gf[0] == pytest.approx(dF, rel=1e-9)
    _, dT, _ = orc.drag_tangent(*args, boundary="sbb", dtau=1.0)
    assert abs(gt - dT) <= 1e-12
    du = workloads.fourier_velocity_field(c["shape"], 3, 1.0, 5)
    _, dU, _ = orc.drag_tangent(*args, boundary="sbb", du0=du)
    assert float((gu * du).sum()) == pytest.approx(dU, rel=1e-9)
    sim.close()


def test_autograd_function(lib):
    """torch.autograd through mean_drag gives the ABI's gradients, scaled by
    the incoming gradient."""
    import torch
    c = SMALL
    u0 = workloads.fourier_velocity_field(c["shape"], 2, 1e-2, 21)
    sim = make_sim(lib, c["shape"], c["pos"], c["diameter"], c["tau"], "fp64")
    J0, gt0, gf0, gu0 = run(lib, sim, c["tau"], (c["force"], 0, 0), u0, c["steps"], 10)
    tau = torch.tensor(c["tau"], dtype=torch.float64, requires_grad=True)
    force = torch.tensor([c["force"], 0.0, 0.0], dtype=torch.float64, requires_grad=True)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda", requires_grad=True)
    J = sim.mean_drag(tau, force, u, c["steps"], 10)
    (3.0 * J).backward()
    assert J.item() == J0
    assert tau.grad.item() == pytest.approx(3 * gt0, rel=1e-15)
    assert np.allclose(force.grad.numpy(), 3 * gf0, rtol=1e-15, atol=0)
    assert np.allclose(u.grad.cpu().numpy(), 3 * gu0, rtol=1e-15, atol=0)
    sim.close()


def test_errors(lib):
    c = SMALL
    sim = lib.Simulation(c["shape"], precision="fp64", tau=0.7)
    sim.add_sphere(c["pos"], c["diameter"], 0.5)   # free sphere: no adjoint
    u0 = np.zeros((3,) + tuple(reversed(c["shape"])))
    with pytest.raises(lib.LbmpError) as e:
        run(lib, sim, 0.7, (0, 0, 0), u0, 4, 2)
    assert e.value.status == 7   # unsupported
    sim.close()
    sim = make_sim(lib, c["shape"], c["pos"], c["diameter"], 0.7, "fp64")
    import torch
    one = torch.ones((), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.LbmpError) as e:
        lib.lbmp_drag_backward(sim.h, one.data_ptr(), 0, 0, 0)
    assert e.value.status == 1
    sim.close()


def test_full_workload_fp32_against_fp64(orc, lib):
    """The differentiation workload at full size in FP32 (the configuration
    the bench times): J and the initial-velocity gradient (along a seeded
    direction) within 1e-4 of the FP64 tangent oracle, dJ/dtau and dJ/dF_x
    within 1e-4 of FP64 central differences on the GPU's FP64 path."""
    c = workloads.ADJOINT_64
    off = workloads.sub_cell_offset(7)
    pos = tuple(0.5 * n + o for n, o in zip(c["shape"], off))
    u0 = workloads.fourier_velocity_field(c["shape"], c["kmax"], c["amplitude"], 7)
    F = (c["body_force"], 0.0, 0.0)
    s32 = make_sim(lib, c["shape"], pos, c["diameter"], c["tau"], "fp32")
    J, gt, gf, gu = run(lib, s32, c["tau"], F, u0, c["steps"], c["checkpoint"])
    s32.close()
    du = workloads.fourier_velocity_field(c["shape"], 3, 1.0, 8)
    Jo, dU, _ = orc.drag_tangent(c["shape"], c["tau"], pos, c["diameter"], c["steps"], u0=u0, body_force=F, du0=du)
    assert J == pytest.approx(Jo, rel=1e-4)
    assert float((gu * du).sum()) == pytest.approx(dU, rel=1e-4)
    # FP64 central differences on the GPU for tau and F_x
    s64 = make_sim(lib, c["shape"], pos, c["diameter"], c["tau"], "fp64")

    def J64(tau, fx):
        return forward(lib, s64, tau, (fx, 0, 0), u0, c["steps"], c["checkpoint"])[0]

    h = 1e-5
    fd_tau = (J64(c["tau"] + h, F[0]) - J64(c["tau"] - h, F[0])) / (2 * h)
    hf = 1e-7
    fd_f = (J64(c["tau"], F[0] + hf) - J64(c["tau"], F[0] - hf)) / (2 * hf)
    s64.close()
    assert gt == pytest.approx(fd_tau, rel=1e-4)
    assert gf[0] == pytest.approx(fd_f, rel=1e-4)


def test_fp64_gradient_u0_element_by_element(orc, lib):
    """dJ/du0 entry by entry against the tangent-linear oracle (one tangent
    run per unit direction): every component of every fluid cell next to the
    sphere (where the reverse step takes the link rules, k_adj_near), of 64
    seeded fluid cells elsewhere, and of 8 cells inside the sphere (zero: the
    fluid there is dropped).  16^3, d = 5, 20 steps, checkpoints every 7."""
    shape, pos, D, tau, steps = (16, 16, 16), (8.3, 7.6, 8.2), 5.0, 0.7, 20
    F = (1e-5, 2e-6, 0.0)
    u0 = workloads.fourier_velocity_field(shape, 2, 1e-2, 31)
    sim = make_sim(lib, shape, pos, D, tau, "fp64")
    J, _, _, gu = run(lib, sim, tau, F, u0, steps, 7)
    flags = sim.flags().reshape(tuple(reversed(shape)))
    sim.close()
    from lattice_ref import C
    solid = flags != 0
    near = np.zeros_like(solid)
    for c in C[1:]:
        near |= np.roll(solid, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2))
    near &= ~solid
    rng = np.random.default_rng(7)
    far = np.argwhere(~solid & ~near)
    cells = [tuple(v) for v in np.argwhere(near)]
    cells += [tuple(v) for v in far[rng.choice(len(far), 64, replace=False)]]
    inside = np.argwhere(solid)
    cells += [tuple(v) for v in inside[rng.choice(len(inside), 8, replace=False)]]
    assert np.count_nonzero(near) >= 50
    scale = np.abs(gu).max()
    worst = 0.0
    for (z, y, x) in cells:
        for a in range(3):
            du = np.zeros_like(u0)
            du[a, z, y, x] = 1.0
            _, d, _ = orc.drag_tangent(shape, tau, pos, D, steps, u0=u0, body_force=F, du0=du)
            worst = max(worst, abs(gu[a, z, y, x] - d))
            if solid[z, y, x]:
                assert gu[a, z, y, x] == 0.0 and d == 0.0
    assert worst <= 1e-9 * scale, worst / scale
