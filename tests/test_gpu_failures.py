"""Failure handling through the C ABI, on the GPU, without faulting it.

- Allocation failure: an allocator callback that returns NULL on its k-th
  call, for every k that a uniform and a refined workflow reach (create,
  sphere, fluid, steps, a rebuilt hierarchy): the call that needed the
  memory returns LBMP_ERR_OOM, nothing is launched on a missing buffer, and
  destroying the handle returns every block the callback handed out.
- Instability: a plain-MEM sphere far lighter than the stability limit
  drives the device status word to LBMP_ERR_UNSTABLE within a few steps; the
  error text says so, the handle is still destroyed cleanly and the next
  handle on the device runs normally.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L
    L._native.load()
    return L


class _Counting:
    """Allocator callbacks over PyTorch's caching allocator that refuse the
    fail_at-th request (0: none) and keep the live blocks."""

    def __init__(self, native, torch, device, stream, fail_at):
        self.calls = 0
        self.live = {}

        def _alloc(nbytes, ctx):
            self.calls += 1
            if self.calls == fail_at:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream))
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, nbytes, ctx):
            self.live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = native.ALLOC_FN(_alloc)
        self.free = native.FREE_FN(_free)


def _uniform_flow(L):
    return [
        ("create", lambda s: L.Simulation((32, 32, 32), precision="fp32", tau=0.6)),
        ("sphere", lambda s: s.add_sphere((16.3, 15.8, 16.4), 8.0, 0.5, cv=0.5)),
        ("gravity", lambda s: s.set_gravity((0, 0, -2.5e-5))),
        ("fluid", lambda s: s.init_fluid(u_field=np.zeros((3, 32, 32, 32)))),
        ("step", lambda s: s.step(3)),
        ("links", lambda s: s.links()),
    ]


def _refined_flow(L):
    return [
        ("create", lambda s: L.Simulation((16, 16, 32), precision="fp32", tau=0.7, levels=3,
                                          bc=("noslip", "noslip", "periodic"))),
        ("sphere", lambda s: s.add_sphere((32.3, 31.6, 60.2), 10.0, 0.5, cv=0.5)),
        ("gravity", lambda s: s.set_gravity((0, 0, -1e-4))),
        ("fluid", lambda s: s.init_fluid()),
        ("step", lambda s: s.step(2)),
        ("rebuild", lambda s: s.refine_box((8, 8, 100), (40, 40, 120))),
        ("step", lambda s: s.step(1)),
        ("cells", lambda s: s.level_cells(2)),
    ]


def _run(flow):
    """Runs the calls in order; returns (handle or None, name of the call that
    failed or None, its error)."""
    s = None
    for name, call in flow:
        try:
            r = call(s)
        except Exception as e:   # noqa: BLE001 -- the test inspects it
            return s, name, e
        if name == "create":
            s = r
    return s, None, None


@pytest.mark.parametrize("flow", [_uniform_flow, _refined_flow])
def test_allocation_failure_reports_oom_and_frees_everything(lib, monkeypatch, flow):
    import torch
    made = []

    def factory(device, stream, fail_at):
        a = _Counting(lib._native, torch, device, stream, fail_at)
        made.append(a)
        return a

    monkeypatch.setattr(lib, "_TorchAllocator", lambda device, stream: factory(device, stream, 0))
    s, name, err = _run(flow(lib))
    assert err is None, (name, err)
    total = made[-1].calls
    s.close()
    assert total >= 8 and not made[-1].live
    for k in range(1, total + 1):
        monkeypatch.setattr(lib, "_TorchAllocator", lambda device, stream, k=k: factory(device, stream, k))
        s, name, err = _run(flow(lib))
        assert isinstance(err, lib.LbmpError) and err.status == 2, (k, name, err)   # LBMP_ERR_OOM
        if s is not None and name == "rebuild":
            # a hierarchy left half-built refuses every further call before launching anything
            with pytest.raises(lib.LbmpError) as again:
                s.step(1)
            assert again.value.status == 2
        if s is not None:
            s.close()
        assert not made[-1].live, (k, name, "blocks not returned")
    torch.cuda.synchronize()


def test_unstable_light_sphere_sets_status_and_handle_recovers(lib):
    s = lib.Simulation((64, 64, 128), precision="fp32", tau=0.5 + 3 * 0.01 * 10 / 100)
    s.add_sphere((32.0, 32.0, 6.0), 10.0, 0.02, cv=0.0)   # plain MEM, far below the limit (about 0.26 at d = 10)
    s.set_ga(100.0, 0.01, (0.0, 0.0, -1.0))
    s.init_fluid()
    with pytest.raises(lib.LbmpError) as e:
        s.step(200)
    assert e.value.status == 4   # LBMP_ERR_UNSTABLE
    assert "unstable" in lib.lbmp_last_error(s.h).lower() or "unstable" in str(e.value).lower()
    s.close()
    t = lib.Simulation((32, 32, 32), precision="fp32", tau=0.6)
    t.add_sphere((16.3, 15.8, 16.4), 8.0, 0.5, cv=0.5)
    t.set_gravity((0, 0, -2.5e-5))
    t.init_fluid()
    t.step(20)
    assert np.all(np.isfinite(t.particle()))
    t.close()
