"""The allocation-free boundary-cell entry point against the library's own list.

lbmp_boundary_cells_noalloc exists for callers that cannot allocate device
memory (a host function enqueued on a stream, a loop that must not risk the
device synchronisation an allocation may bring, a process whose device
memory is owned by another allocator).  Its scratch is a fixed device array
inside the library.  This test calls it through the C ABI twice in a row (the
sphere moves in between) and checks that it returns exactly the boundary-cell
list the coupled step built for itself, which lbmp_get_links exposes.  The
file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ordered_unique(a):
    _, first = np.unique(a, return_index=True)
    return a[np.sort(first)]


def test_noalloc_boundary_cells_match_coupled_step():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L

    shape = (48, 40, 56)
    sim = L.Simulation(shape, precision="fp32", tau=0.6)
    sim.add_sphere((23.7, 19.2, 20.4), 12.0, 0.5, cv=0.5)
    sim.set_gravity((0.0, 0.0, -4e-4))
    sim.set_particle_velocity((0.02, -0.01, 0.05))
    sim.init_fluid()
    stream = torch.cuda.current_stream()
    cap = 4096
    for call in range(2):
        if call == 1:
            sim.step(25)   # the sphere moves: a different list
        flags_host = sim.flags()
        flags = torch.from_numpy(flags_host).cuda()
        out = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        centre = sim.particle()[6:9]
        L.lbmp_boundary_cells_noalloc(flags.data_ptr(), shape, (1, 1, 1), centre, 12.0, out.data_ptr(), cap,
                                      count.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        n = int(count.item())
        got = out[:n].cpu().numpy().astype(np.int64)
        cells, _, _ = sim.links()
        expect = _ordered_unique(cells)
        assert n == len(expect) > 0
        assert np.array_equal(got, expect)
        assert np.all(out[n:].cpu().numpy() == -1)
    # a sphere whose box exceeds the fixed scratch (68^3 cells > 64^3) is
    # refused on the host before any kernel runs or any pointer is read
    with pytest.raises(L.LbmpError) as e:
        L.lbmp_boundary_cells_noalloc(flags.data_ptr(), (128, 128, 128), (1, 1, 1), (64.0, 64.0, 64.0), 60.0,
                                      out.data_ptr(), cap, count.data_ptr(), stream.cuda_stream)
    assert "scratch" in str(e.value)
    sim.close()
