"""Host logic of the Tolman sweep driver (no GPU): the box sides of the radius
sweep and the test that decides which droplets enter the Eq. sigma_c fit."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tolman():
    # tolman.py imports the binding, which needs the built library; load it only if present
    sys.path.insert(0, ROOT)
    if importlib.util.find_spec("torch") is None:
        pytest.skip("needs torch")
    build = importlib.import_module("paper_2112_02574_gb300.build")
    if not os.path.exists(build.LIB):
        pytest.skip("library not built")
    from paper_2112_02574_gb300 import tolman as T

    return T


def test_droplet_side_is_about_4R_and_a_multiple_of_4(tolman):
    for R in (8.0, 8.01, 10.13, 12.5, 40.0):
        L = tolman.droplet_side(R)
        assert L % 4 == 0 and 4 * R <= L < 4 * R + 4


def test_usable_droplet_criteria(tolman):
    good = {"dP": 0.02, "R": 10.0, "R_s": 10.3, "dP_change": 5e-6}
    assert tolman.usable(good)
    assert not tolman.usable({**good, "dP": -1e-4})  # no pressure jump: not a droplet
    assert not tolman.usable({**good, "R_s": -4.9})  # interface wider than the droplet
    assert not tolman.usable({**good, "R_s": 283.0})  # dissolved
    assert not tolman.usable({**good, "dP_change": 2e-3})  # not settled
    assert tolman.usable({**good, "dP_change": 2e-3}, max_change=1e-2)
