"""Host-side checks of the autotuner's candidate lists (no GPU): every candidate
it would time is a configuration the library accepts, the library default comes
first, and the staged candidates appear exactly where the library would run the
staged kernel."""
import pytest


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2112_02574_gb300 import binding

    return binding


CASES = [
    # (shape, lattice, stencil, storage name, staged eligible)
    ((128, 128, 128), 1, 0, "F32", True),
    ((96, 40, 64), 1, 0, "F16", True),
    ((36, 20, 24), 1, 0, "BF16", True),
    ((70, 9, 6), 1, 0, "F32", True),
    ((37, 11, 19), 1, 0, "F32", False),   # odd nx: no whole 16-byte chunks of FP32 pairs
    ((37, 11, 19), 1, 0, "F64", True),    # FP64: one site per chunk
    ((34, 10, 16), 1, 0, "F16", False),   # nx not a multiple of 4
    ((64, 64, 256), 1, 1, "F32", False),  # E6: generic kernel only
    ((64, 64, 1), 0, 0, "F32", False),    # D2Q9
]


@pytest.mark.parametrize("shape,lattice,stencil,storage,eligible", CASES)
def test_candidates_are_valid(B, shape, lattice, stencil, storage, eligible):
    from paper_2112_02574_gb300 import tune

    st = getattr(B, f"SC_STORE_{storage}")
    p = B.make_params(shape, lattice=lattice, stencil=stencil, storage=st, tau=(1.0, 1.0), G=2.5)
    assert tune.staged_eligible(p) == eligible
    cands = tune.candidates_for(p)
    assert cands[0] == (0, 0, 0, 0, 0)
    assert any(c[0] == 2 for c in cands) == eligible
    for variant, ty, tz, ns, mb in cands:
        q = B.make_params(shape, lattice=lattice, stencil=stencil, storage=st, tau=(1.0, 1.0), G=2.5, tile_y=ty,
                          tile_z=tz, variant=variant, stages=ns, blocks_per_sm=mb)
        assert B.sc_workspace_bytes(q) > 0, ((variant, ty, tz, ns, mb), B.sc_last_error())
