"""The oracle against its stored expected values (tests/golden/, written by
tests/golden/make_golden.py, which runs the oracle only). A change to the
oracle's arithmetic, its random-number layout or its window loop shows up
here; the stored tau is also the closed form for this mesh (a regular Kuhn
grid of 0.5 um cubes with D = 1e-11 m^2/s)."""
import importlib.util
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)


@pytest.mark.parametrize("prec", [32, 64])
def test_oracle_reproduces_stored_cuboid_run(prec):
    ref = golden.read(os.path.join(HERE, "golden", f"cuboid_prec{prec}.txt"))
    w, o = golden.cuboid(prec)
    assert o.windows == ref["windows"] == 14
    assert o.tau == ref["tau"]
    c = o.get_counts()
    assert np.array_equal(c, ref["counts"])
    assert c.sum(axis=1).tolist() == ref["totals"]
    # A + C and B + C are conserved by A + B <-> C
    assert ref["totals"][0] + ref["totals"][2] == 5000 and ref["totals"][1] + ref["totals"][2] == 5000


def test_stored_tau_is_the_closed_form():
    """tau = h^2 / (D (24 + 4 sqrt 6)) on a regular Kuhn grid of cube edge h."""
    ref = golden.read(os.path.join(HERE, "golden", "cuboid_prec32.txt"))
    h, D = 0.5e-6, 1e-11
    assert math.isclose(ref["tau"], h * h / (D * (24 + 4 * math.sqrt(6))), rel_tol=1e-12)
