"""lbc_fbar_moments_noalloc: the allocation-free moment sums agree with the
box's own invariants.

This entry point exists for callers that cannot allocate device memory
(processes whose memory is fully reserved by a pool or another framework,
hooks holding another owner's buffer); it keeps its scratch in a fixed
device array.  The test calls it through the C ABI on a
device copy of the populations and compares, on two calls in a row, with
lbc_box_invariants (the existing entry point, which uses the box's arena)
within the FP64 tolerance used by the other parity tests.  Kept in a file of
its own, collected last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _noalloc_moments(lib, fbar, shape):
    import torch
    nz, ny, nx = shape
    dev = torch.from_numpy(np.ascontiguousarray(fbar)).to("cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.lbc_fbar_moments_noalloc(C.c_void_p(dev.data_ptr()), nx, ny, nz,
                                      C.c_void_p(out.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    assert st == 0, st
    return out.cpu().numpy()


def test_noalloc_moments_match_box_invariants_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_1406_2211_gb300 import lbc
    lib = lbc.library()
    shape = (12, 10, 9)
    nz, ny, nx = shape
    lat = lbc.lattice_desc(nx, ny, nz, collision="mrt", tau=0.8, storage="f64")
    box = lbc.Box(lat)
    box.set_populations(synth.random_populations(shape, seed=17, amp=1e-2))
    for nsteps in (3, 5):               # two calls in a row, different states
        box.step(nsteps)
        mass, mom, st = box.invariants()
        assert st == 0
        got = _noalloc_moments(lib, box.get_populations(), shape)
        assert abs(got[0] - mass) < 1e-12 * mass
        assert np.abs(got[1:] - mom).max() < 1e-12
    box.close()


def test_noalloc_rejects_oversized_and_null():
    import torch
    from paper_1406_2211_gb300 import lbc
    lib = lbc.library()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    buf = torch.zeros(19, dtype=torch.float64, device="cuda")
    too_deep = lbc.LBC_NOALLOC_MAX_PLANES + 1
    assert lib.lbc_fbar_moments_noalloc(C.c_void_p(buf.data_ptr()), 1, 1, too_deep,
                                        C.c_void_p(out.data_ptr()), None) == lbc.LBC_ERR_ARG
    assert lib.lbc_fbar_moments_noalloc(None, 1, 1, 1, C.c_void_p(out.data_ptr()),
                                        None) == lbc.LBC_ERR_ARG


def test_noalloc_deepest_array_uses_every_scratch_slot():
    """nz = LBC_NOALLOC_MAX_PLANES (the last scratch slot written), on a
    1 x 1 x nz column whose planes carry different sums, against the
    existing entry point's invariants, twice in a row."""
    import torch
    from paper_1406_2211_gb300 import lbc
    lib = lbc.library()
    nz = lbc.LBC_NOALLOC_MAX_PLANES
    shape = (nz, 1, 1)
    lat = lbc.lattice_desc(1, 1, nz, collision="bgk", tau=0.9, storage="f64")
    box = lbc.Box(lat)
    box.set_populations(synth.random_populations(shape, seed=23, amp=1e-2))
    for nsteps in (1, 2):
        box.step(nsteps)
        mass, mom, st = box.invariants()
        assert st == 0
        got = _noalloc_moments(lib, box.get_populations(), shape)
        assert abs(got[0] - mass) < 1e-12 * mass
        assert np.abs(got[1:] - mom).max() < 1e-12
    box.close()
