"""GPU test of the failure path of the step kernel's bounded wait for its
bulk copies: a wait that nothing completes gives up after its cycle limit
and reports STEPS_ERR_TIMEOUT through the error word, without a fault, a
trap or a hang, and the device stays usable for the next call. The same
wait completes when the copy is delivered."""
import numpy as np
import pytest

import oracle
from paper_1610_02258_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import capi as c
    return c


def test_bounded_wait_completes_and_times_out(capi):
    capi.steps_debug_wait(True, 1 << 24)           # the copy arrives: no error
    for limit in (1 << 12, 1 << 20):
        with pytest.raises(capi.StepsError) as e:
            capi.steps_debug_wait(False, limit)    # nothing arrives: the limit runs out
        assert e.value.code == -6 and "did not complete" in str(e.value)
    with pytest.raises(capi.StepsError) as e:
        capi.steps_debug_wait(False, 0)
    assert e.value.code == -1
    # the device is still usable: a small run equals the oracle
    w = I.config1()
    g = capi.from_workload(w)
    g.run(w.t_end)
    o = oracle.from_workload(w, prec=32)
    o.run(w.t_end)
    assert np.array_equal(g.get_counts(), o.get_counts())
