"""CPU checks of the C ABI: the library builds, loads without a GPU, and
exports every entry point that include/sph.h declares; the binding names the
same set."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1702_07760_gb300 import build as B
from paper_1702_07760_gb300 import sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(headers=("sph.h", "sph_surrogate.h")):
    names = set()
    for h in headers:
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sph.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm
    out = subprocess.run(["nm", "-D", "--defined-only", sph.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sph_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_the_header(lib):
    assert sorted(sph.EXPORTS) == declared()


def test_invalid_parameters_are_rejected_without_a_gpu(lib):
    from paper_1702_07760_gb300 import workloads as WL
    w = WL.drop_tank(2, (4, 4))
    bad = dict(w.params, gamma=5.0)
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(bad, w.x, w.u, w.rho, w.phase, w.wall)
    assert e.value.code == -1 and "gamma" in str(e.value)
    bad = dict(w.params, cell_size=w.params["h"])
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(bad, w.x, w.u, w.rho, w.phase, w.wall)
    assert e.value.code == -1
    x = w.x.copy()
    x[0, 0] = w.params["box_hi"][0] + 1.0
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(w.params, x, w.u, w.rho, w.phase, w.wall)
    assert e.value.code == -1 and "outside" in str(e.value)
    ph = w.phase.copy()
    wl = w.wall.copy()
    ph[wl == 1] = 1
    with pytest.raises(sph.SphError):
        sph.Simulation(w.params, w.x, w.u, w.rho, ph, wl)
    # the boundary-reading switch is 0 or 1, the reserved word 0
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(dict(w.params, renorm_walls=2), w.x, w.u, w.rho, w.phase, w.wall)
    assert e.value.code == -1 and "renorm_walls" in str(e.value)
    prm = sph.make_params(w.params)
    prm.reserved = 1
    h = C.c_void_p()
    rc = lib.sph_create(C.byref(prm), w.n, sph._dp(w.x), sph._dp(w.u), sph._dp(w.rho),
                        w.phase.ctypes.data_as(C.POINTER(C.c_uint8)), w.wall.ctypes.data_as(C.POINTER(C.c_uint8)),
                        None, C.byref(h))
    assert rc == -1 and "reserved" in lib.sph_last_error().decode() and not h.value


def test_fp32_peak_rejects_bad_arguments_without_a_gpu(lib):
    t, m = C.c_double(), C.c_double()
    assert lib.sph_fp32_peak(0, 16, None, C.byref(t), C.byref(m)) == -1
    assert lib.sph_fp32_peak(9, 16, None, C.byref(t), C.byref(m)) == -1
    assert lib.sph_fp32_peak(8, 0, None, C.byref(t), C.byref(m)) == -1
    assert lib.sph_fp32_peak(8, 16, None, None, C.byref(m)) == -1


def test_null_handles_are_rejected_without_a_gpu(lib):
    """Entry points taking a handle return SPH_EINVAL for NULL before any
    CUDA call."""
    import ctypes as C
    dp = C.POINTER(C.c_double)
    buf = (C.c_double * 8)()
    p = C.cast(buf, dp)
    assert lib.sph_advance_host(None, 1e-5, 1, p, p, p, p, p, p) == -1
    assert lib.sph_read_state(None, p, p, p) == -1
    assert lib.sph_set_state(None, p, p, p) == -1
    assert lib.sph_run(None, 1e-5, 1, 1) == -1
    counts = (C.c_int64 * 4)()
    assert lib.sph_pair_classes(None, counts) == -1
    assert lib.sph_pair_stats(None, counts) == -1


def test_kernels_compile_for_sm103a_without_spills():
    out = subprocess.run(B.nvcc_command("/tmp/libsph_probe.so", ("-Xptxas", "-v")),
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-2000:]
    info = out.stderr
    for kern in ("k_sweep_b",):
        blocks = [b for b in info.split("Function properties for ") if kern in b.split("\n")[0]]
        assert blocks, kern
        for b in blocks:
            assert "0 bytes spill stores" in b, b[:400]


def test_batch_validation_without_a_gpu(lib):
    """sph_create_batch checks the shared parameters and every instance's
    particles before it touches the device."""
    from paper_1702_07760_gb300 import workloads as WL
    ws = WL.drop_batch_2d(k=3, seed=5, d_range=(4.0, 5.0))
    # instances differing in a shared parameter (h through dx)
    odd = WL.drop_tank(2, (8, 16), dx=3e-4)
    with pytest.raises(sph.SphError) as e:
        sph.Simulation.batch(ws + [odd])
    assert e.value.code == -1 and "share" in str(e.value)
    # a particle outside its own instance's box
    bad = ws[1].copy()
    bad.x[0, 1] = bad.params["box_hi"][1] + 1e-3
    with pytest.raises(sph.SphError) as e:
        sph.Simulation.batch([ws[0], bad, ws[2]])
    assert e.value.code == -1 and "outside" in str(e.value)
    bad = ws[2].copy()
    bad.params = dict(bad.params, gamma=6.0)
    with pytest.raises(sph.SphError) as e:
        sph.Simulation.batch([ws[0], bad])
    assert e.value.code == -1


def test_periodic_and_piston_validation_without_a_gpu(lib):
    """Periodic axes and piston flags are checked before the device is touched."""
    from paper_1702_07760_gb300 import workloads as WL
    w = WL.wave_tank_small()
    p = w.params
    # a period that is not a whole number of super-cells
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(dict(p, cell_size=p["cell_size"] * 1.07), w.x, w.u, w.rho, w.phase, w.wall)
    assert e.value.code == -1 and "periodic" in str(e.value)
    # a periodic bit beyond dim
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(dict(p, periodic=8), w.x, w.u, w.rho, w.phase, w.wall)
    assert e.value.code == -1
    # wall flags other than 0, 1, 2; an oil piston
    wl = w.wall.copy()
    wl[0] = 3
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(p, w.x, w.u, w.rho, w.phase, wl)
    assert e.value.code == -1 and "piston" in str(e.value)
    ph = w.phase.copy()
    ph[w.wall == 2] = 1
    with pytest.raises(sph.SphError):
        sph.Simulation(p, w.x, w.u, w.rho, ph, w.wall)
    # no periodic axes in a batch
    ws = WL.drop_batch_2d(k=2, seed=5, d_range=(4.0, 5.0))
    per = [v.copy() for v in ws]
    for v in per:
        v.params = dict(v.params, periodic=1)
    with pytest.raises(sph.SphError) as e:
        sph.Simulation.batch(per)
    assert e.value.code == -1 and "batch" in str(e.value)
