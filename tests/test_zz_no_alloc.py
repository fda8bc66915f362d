"""The allocation-free boundary-cell entry point against the library's own list.

lbmp_boundary_cells_noalloc exists for callers that cannot allocate device
memory (a loop that must not risk the device synchronisation an allocation
may bring, a process whose device memory is owned by another allocator).
Its scratch is a fixed device array inside the library.  This test calls it
through the C ABI twice in a row (the sphere moves in between) and checks
that it returns exactly the boundary-cell list the coupled step built for
itself, which lbmp_get_links exposes: on a periodic grid, and on a grid with
walls on two axes and the sphere near one of them.  The file is named to be
collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ordered_unique(a):
    _, first = np.unique(a, return_index=True)
    return a[np.sort(first)]


def _check_against_coupled_step(L, torch, shape, bc, periodic, pos, d, vel, steps):
    sim = L.Simulation(shape, precision="fp32", tau=0.6, bc=bc)
    sim.add_sphere(pos, d, 0.5, cv=0.5)
    sim.set_gravity((0.0, 0.0, -4e-4))
    sim.set_particle_velocity(vel)
    sim.init_fluid()
    stream = torch.cuda.current_stream()
    cap = 4096
    for call in range(2):
        if call == 1:
            sim.step(steps)   # the sphere moves: a different list
        flags_host = sim.flags()
        flags = torch.from_numpy(flags_host).cuda()
        out = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        centre = sim.particle()[6:9]
        L.lbmp_boundary_cells_noalloc(flags.data_ptr(), shape, periodic, centre, d, out.data_ptr(), cap,
                                      count.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        n = int(count.item())
        got = out[:n].cpu().numpy().astype(np.int64)
        cells, _, _ = sim.links()
        expect = _ordered_unique(cells)
        assert n == len(expect) > 0
        assert np.array_equal(got, expect)
        assert np.all(out[n:].cpu().numpy() == -1)
    sim.close()
    return flags, out, count, stream


def test_noalloc_boundary_cells_match_coupled_step():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L

    flags, out, count, stream = _check_against_coupled_step(
        L, torch, (48, 40, 56), ("periodic",) * 3, (1, 1, 1), (23.7, 19.2, 20.4), 12.0, (0.02, -0.01, 0.05), 25)
    # walls on x and y, the sphere two cells from the x = 0 wall and its box
    # wider than the y extent (the coupled step then starts that box at 0)
    _check_against_coupled_step(L, torch, (40, 18, 48), ("noslip", "noslip", "periodic"), (0, 0, 1),
                                (8.3, 9.1, 24.6), 12.0, (-0.01, 0.0, 0.03), 20)
    # a sphere whose box exceeds the fixed scratch (68^3 cells > 64^3) is
    # refused on the host before any kernel runs or any pointer is read
    with pytest.raises(L.LbmpError) as e:
        L.lbmp_boundary_cells_noalloc(flags.data_ptr(), (128, 128, 128), (1, 1, 1), (64.0, 64.0, 64.0), 60.0,
                                      out.data_ptr(), 4096, count.data_ptr(), stream.cuda_stream)
    assert "scratch" in str(e.value)
