"""The allocation-free cell sort (sph_cell_sort_noalloc) against the regular
cell-list build.

sph_cell_sort_noalloc is for callers that cannot allocate device memory (a
host application whose device memory belongs to its own pool or allocator, or
a deployment whose device memory is fixed in advance); its scratch is a fixed
file-scope device array shared by all calls.  Its cell ids and sort order must equal the ones sph_build_cells
produces (integers: bit-exact), on two calls in a row so that the second
call is seen to start from cleared scratch.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1702_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _reference(sph, w):
    sim = sph.Simulation.from_workload(w)
    sim.build_cells()
    cell, order = sim.read("cell"), sim.read("order")
    sim.close()
    return cell, order


def test_noalloc_cell_sort_matches_build_cells():
    import torch

    from paper_1702_07760_gb300 import build as B
    from paper_1702_07760_gb300 import sph

    B.build()
    sph.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    # a 3-D case, then a smaller 2-D case on the same scratch
    cases = [WL.drop_tank(3, (24, 20, 36), drop_d_dx=8, seed=21, perturb=True),
             WL.drop_tank(2, (37, 53), drop_d_dx=9, seed=22, quantise=16)]
    for w in cases:
        ref_cell, ref_order = _reference(sph, w)
        x_dev = torch.tensor(w.x, dtype=torch.float64, device="cuda")
        cell_dev = torch.full((w.n,), -7, dtype=torch.int32, device="cuda")
        order_dev = torch.full((w.n,), -7, dtype=torch.int32, device="cuda")
        sph.cell_sort_noalloc(w.params, w.n, x_dev.data_ptr(), cell_dev.data_ptr(), order_dev.data_ptr(),
                              stream.cuda_stream)
        assert np.array_equal(cell_dev.cpu().numpy(), ref_cell)
        assert np.array_equal(order_dev.cpu().numpy(), ref_order)


def test_noalloc_cell_sort_rejects_sizes_beyond_its_limit():
    from paper_1702_07760_gb300 import build as B
    from paper_1702_07760_gb300 import sph

    B.build()
    w = WL.drop_tank(2, (8, 8))
    with pytest.raises(sph.SphError) as e:
        sph.cell_sort_noalloc(w.params, (1 << 20) + 1, 0, 0, 0)
    assert e.value.code == -1 and "2^20" in str(e.value)
    big = dict(w.params, cell_size=w.params["cell_size"] * 1e-3)
    with pytest.raises(sph.SphError) as e:
        sph.cell_sort_noalloc(big, 16, 0, 0, 0)
    assert e.value.code == -1 and "cells" in str(e.value)


def test_noalloc_cell_sort_reports_a_particle_outside_the_box():
    """A particle beyond box_hi: the hash clamps its cell into the grid (every
    access stays in bounds), raises the out-of-box flag, and the call returns
    SPH_EDOMAIN; the next call with the particle back inside succeeds and
    matches sph_build_cells."""
    import torch

    from paper_1702_07760_gb300 import build as B
    from paper_1702_07760_gb300 import sph

    B.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    w = WL.drop_tank(2, (20, 30), drop_d_dx=6, seed=23, quantise=16)
    x = w.x.copy()
    x[5, 0] = w.params["box_hi"][0] + 10 * w.params["cell_size"]
    x_dev = torch.tensor(x, dtype=torch.float64, device="cuda")
    cell_dev = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    order_dev = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SphError) as e:
        sph.cell_sort_noalloc(w.params, w.n, x_dev.data_ptr(), cell_dev.data_ptr(), order_dev.data_ptr(),
                              stream.cuda_stream)
    assert e.value.code == -6
    x_dev = torch.tensor(w.x, dtype=torch.float64, device="cuda")
    sph.cell_sort_noalloc(w.params, w.n, x_dev.data_ptr(), cell_dev.data_ptr(), order_dev.data_ptr(),
                          stream.cuda_stream)
    ref_cell, ref_order = _reference(sph, w)
    assert np.array_equal(cell_dev.cpu().numpy(), ref_cell)
    assert np.array_equal(order_dev.cpu().numpy(), ref_order)
