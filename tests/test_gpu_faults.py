"""Failure detection on the device without a GPU fault: the bounded wait that
every kernel of the library uses on its mbarriers (TMA arrivals, tensor-core
commits) gives up when nothing completes the barrier, reports BD_ERR_TIMEOUT
to the host, and leaves the CUDA context usable for the next call."""
import ctypes
import time

import numpy as np
import pytest

from paper_2208_06559_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bd():
    from paper_2208_06559_gb300 import build as b
    b.build()
    import paper_2208_06559_gb300 as pkg
    pkg.lib()
    return pkg


def test_bounded_wait_gives_up_and_the_context_stays_usable(bd):
    L = bd.lib()
    st = ctypes.c_int(123)
    assert L.bd_selftest_bounded_wait(1, ctypes.byref(st)) == bd.binding.BD_OK
    assert st.value == bd.binding.BD_OK            # the phase completed at once
    t0 = time.perf_counter()
    assert L.bd_selftest_bounded_wait(0, ctypes.byref(st)) == bd.binding.BD_OK
    waited = time.perf_counter() - t0
    assert st.value == bd.binding.BD_ERR_TIMEOUT   # nothing arrived: the wait gave up
    assert 0.3 < waited < 30.0, waited
    # the same context runs the next work: a mixed step and an FP64 step
    Nc = np.array([40, 23], np.int32)
    r0 = torch.from_numpy(inputs.random_walk(Nc, 91)).cuda()
    noise = torch.from_numpy(inputs.gaussian_noise(2, int(Nc.sum()), 92)).cuda()
    for prec in (bd.MIXED_TF32, bd.FP64):
        with bd.Context(Nc, precision=prec, flow=1, Wi=10.0) as ctx:
            ctx.set_state(r0)
            ctx.step(noise)
            obs, st_c = ctx.observables()
            assert (st_c == 0).all()
            assert obs[:, bd.OBS_MAXDEV].max().item() < 1e-10
