"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/sc.h declares, and rejects invalid arguments with
SC_EINVAL before touching any device memory."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2112_02574_gb300 import binding

    return binding


def test_every_declared_symbol_is_exported(B):
    names = B.declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(B.lib, n), n
        assert hasattr(B, n), f"binding lacks {n}"


def test_workspace_bytes_layout(B):
    p = B.make_params((128, 128, 128), storage=B.SC_STORE_F32)
    ws = B.sc_workspace_bytes(p)
    pops = 2 * 2 * 19 * 128**3 * 4
    assert ws >= pops + 4 * 8 * 128**3
    assert ws % 256 == 0
    p16 = B.make_params((128, 128, 128), storage=B.SC_STORE_F16)
    # 16-bit pairs plus one FP32 reference-density pair per site in each of the two buffers
    assert B.sc_workspace_bytes(p16) - ws == 2 * 2 * 19 * 128**3 * 2 - pops + 2 * 8 * 128**3


@pytest.mark.parametrize("bad", [
    dict(shape=(0, 4, 4)),
    dict(shape=(4, 4, 4), lattice=7),
    dict(shape=(4, 4, 2), lattice=0),            # D2Q9 with nz != 1
    dict(shape=(4, 4, 1), lattice=0, stencil=1),  # E6 on D2Q9
    dict(shape=(4, 4, 4), tau=(0.5, 1.0)),
    dict(shape=(4, 4, 4), tau=(1.0, float("nan"))),
    dict(shape=(4, 4, 4), storage=9),
    dict(shape=(4, 4, 4), tile_y=3),
    dict(shape=(4, 4, 4), G=float("inf")),
    dict(shape=(64, 4, 4), stages=3),
    dict(shape=(64, 4, 4), tile_y=4, blocks_per_sm=1),
    dict(shape=(64, 4, 4), tile_y=8, stages=2, blocks_per_sm=3),
    dict(shape=(64, 4, 4), tile_y=16, blocks_per_sm=2),
    dict(shape=(64, 4, 4), tile_y=16, stages=2),           # two 32 x 16 FP32 stages do not fit
    dict(shape=(33, 4, 4), tile_y=16),                      # generic kernel (odd nx in FP32): no tile_y 16
    dict(shape=(64, 4, 4), storage=3, tile_y=16),           # F64 staged: tile_y 4 only
])
def test_invalid_parameters_rejected(B, bad):
    shape = bad.pop("shape")
    p = B.make_params(shape, **bad)
    assert B.sc_workspace_bytes(p) == 0
    assert B.sc_last_error() != ""
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(256)
    st = B.lib.sc_create(ctypes.byref(p), dummy, dummy, dummy, 1 << 30, None, ctypes.byref(ctx))
    assert st == B.SC_EINVAL
    assert not ctx.value


def test_null_and_range_arguments(B):
    assert B.lib.sc_step(None, 1) == B.SC_EINVAL
    assert B.lib.sc_sync(None) == B.SC_EINVAL
    assert B.lib.sc_selftest_wait_timeout(None, 16) == B.SC_EINVAL
    assert B.lib.sc_batch_set_persistent(None, 1) == B.SC_EINVAL
    assert B.lib.sc_batch_variant(None) == 0
    assert B.lib.sc_step_config(None, None, 8) == B.SC_EINVAL
    assert B.lib.sc_sigma_minimum(None, 10, None, 3, 1.0, 2.0, 0.1, None, None) == B.SC_EINVAL
    p = B.make_params((8, 8, 8))
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(256)
    # workspace too small -> SC_ENOMEM before any device work
    assert B.lib.sc_create(ctypes.byref(p), dummy, dummy, dummy, 16, None, ctypes.byref(ctx)) == B.SC_ENOMEM
    # misaligned workspace
    assert B.lib.sc_create(ctypes.byref(p), dummy, dummy, ctypes.c_void_p(257), 1 << 30, None,
                           ctypes.byref(ctx)) == B.SC_EINVAL


@pytest.mark.parametrize("bad", [
    dict(shape=(8, 8, 8), psi_self=5),                 # unknown pseudopotential
    dict(shape=(8, 8, 8), G_self=(float("nan"), 0.0)),  # non-finite coupling
    dict(shape=(8, 8, 1), lattice=0, stencil=1),       # E6 on D2Q9
    dict(shape=(2048, 2048, 1024)),                    # more than 2^31 - 1 sites
])
def test_noalloc_profile_applies_the_model_checks(B, bad):
    """The allocation-free profile accepts exactly the parameters sc_create accepts for the model
    (size, lattice, stencil, psi_self, couplings): each of these is SC_EINVAL before any CUDA call."""
    shape = bad.pop("shape")
    p = B.make_params(shape, **bad)
    d = ctypes.c_void_p(256)
    c = (ctypes.c_double * 3)(1.0, 1.0, 0.0)
    assert B.lib.sc_pressure_profile_noalloc(ctypes.byref(p), d, d, 0, c, 0.5, 8, d, None) == B.SC_EINVAL


def test_axis_profile_rejects_more_rows_than_sites(B):
    """The x-axis line holds one site per row: nbins > nx is SC_EINVAL (nbins = nx is accepted as far
    as validation goes; with no GPU the call then fails on the device lookup, not on its arguments)."""
    p = B.make_params((12, 8, 8))
    d = ctypes.c_void_p(256)
    c = (ctypes.c_double * 3)(6.0, 4.0, 4.0)
    assert B.lib.sc_pressure_profile_noalloc(ctypes.byref(p), d, d, B.SC_PROFILE_AXIS_X, c, 1.0, 13, d,
                                             None) == B.SC_EINVAL
    assert "nx" in B.sc_last_error()
    st = B.lib.sc_pressure_profile_noalloc(ctypes.byref(p), d, d, B.SC_PROFILE_AXIS_X, c, 1.0, 12, d, None)
    assert st != B.SC_EINVAL


def test_analysis_entry_points_reject_null_arguments(B):
    c = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    d = ctypes.c_void_p(256)
    assert B.lib.sc_surface_of_tension(None, 0, c, 0.5, 10, 0.0, 0.0, 0.0, d, None) == B.SC_EINVAL
    assert B.lib.sc_diagnostics(None, None, 0, 0.0, d) == B.SC_EINVAL
    p = B.make_params((8, 8, 8))
    # result buffer missing, then a negative step count: both SC_EINVAL before any device work
    assert B.lib.sc_run_host_sigma(ctypes.byref(p), d, d, 10, c, 0.5, 4, None, None, None, d, 1 << 30,
                                   None) == B.SC_EINVAL
    assert B.lib.sc_run_host_sigma(ctypes.byref(p), d, d, -1, c, 0.5, 4, None, None, d, d, 1 << 30,
                                   None) == B.SC_EINVAL
    assert B.lib.sc_run_host_sigma(ctypes.byref(p), d, d, 1, c, 0.5, 4, None, None, d, d, 16,
                                   None) == B.SC_ENOMEM
