"""nrto_solve_noalloc: the batch solve for callers that cannot allocate device memory (real-time loops
that must not pay an allocation's latency, processes whose device memory another allocator holds).
It must give the results of the allocating path (create + nrto_solve) on consecutive calls, whatever
the previous call left in the shared static area, and refuse batches larger than that area."""
import numpy as np
import pytest

from paper_2603_02642_b300 import nrto, workloads as W

from .gpu_common import RTOL64, assert_close

pytestmark = pytest.mark.gpu

OPTS = nrto.Options(rho=10.0, max_inner=60, check=0)
N_OUTER = 3


def _batch_a():
    return [W.unicycle(21, T=30, n_obs=3), W.quadcopter(22, T=20, n_obs=2)]


def _batch_b():
    return [W.quadcopter(23, T=24, n_obs=4), W.arm(24, T=8), W.unicycle(25, T=17, n_obs=5)]


def _allocating(insts, prec=nrto.PREC_FP64):
    prob = nrto.Problem(insts, prec)
    out = prob.solve(OPTS, n_outer=N_OUTER)
    prob.close()
    return out


def _assert_same(got, ref):
    for i in range(len(ref["K"])):
        assert_close(got["u_bar"][i], ref["u_bar"][i], RTOL64, f"u_bar[{i}]")
        assert_close(got["K"][i], ref["K"][i], RTOL64, f"K[{i}]")
    assert_close(got["merit"], ref["merit"], RTOL64, "merit")


def test_noalloc_matches_allocating_path_on_consecutive_calls():
    ref_a, ref_b = _allocating(_batch_a()), _allocating(_batch_b())
    # Same batch twice in a row, then a different batch, then the first again: every call must
    # clear what the previous one left in the shared area.
    _assert_same(nrto.solve_noalloc(_batch_a(), OPTS, N_OUTER), ref_a)
    _assert_same(nrto.solve_noalloc(_batch_a(), OPTS, N_OUTER), ref_a)
    _assert_same(nrto.solve_noalloc(_batch_b(), OPTS, N_OUTER), ref_b)
    _assert_same(nrto.solve_noalloc(_batch_a(), OPTS, N_OUTER), ref_a)


def test_noalloc_mixed_precision_matches_allocating_path():
    insts = _batch_b()
    ref = _allocating(insts, nrto.PREC_MIXED)
    for _ in range(2):
        got = nrto.solve_noalloc(insts, OPTS, N_OUTER, precision=nrto.PREC_MIXED)
        for i in range(len(insts)):
            assert np.array_equal(got["K"][i], ref["K"][i]) and np.array_equal(got["u_bar"][i], ref["u_bar"][i])


def test_noalloc_rejects_batches_beyond_the_static_area():
    big = [W.quadcopter(30 + s, T=100, n_obs=10) for s in range(4)]
    with pytest.raises(nrto.NrtoError) as e:
        nrto.solve_noalloc(big, OPTS, N_OUTER)
    assert e.value.code == 1 and "static device area" in str(e.value)
    # The area is still usable after a refused call.
    _assert_same(nrto.solve_noalloc(_batch_a(), OPTS, N_OUTER), _allocating(_batch_a()))


def test_noalloc_allocates_no_device_memory():
    """After a first call (which looks up the static area and, with lazy module loading, loads the
    kernels it launches), further calls leave the device's free memory unchanged: the call allocates
    nothing.  The library calls the CUDA runtime directly, so any cudaMalloc would show in the
    driver's free-memory count (the torch caching allocator is not involved)."""
    import torch
    nrto.solve_noalloc(_batch_b(), OPTS, N_OUTER)   # every dynamics kind: all FP64 kernels loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for batch in (_batch_a, _batch_b, _batch_a):
        nrto.solve_noalloc(batch(), OPTS, N_OUTER)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_serializes_concurrent_callers():
    """Two host threads calling at once on their own streams: the library's lock serializes the calls
    on the shared area, so both get the results of the allocating path."""
    import threading
    import torch
    ref_a, ref_b = _allocating(_batch_a()), _allocating(_batch_b())
    got = {}
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]

    def run(key, batch, st):
        got[key] = nrto.solve_noalloc(batch, OPTS, N_OUTER, stream=st.cuda_stream)

    ths = [threading.Thread(target=run, args=("a", _batch_a(), streams[0])),
           threading.Thread(target=run, args=("b", _batch_b(), streams[1]))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    _assert_same(got["a"], ref_a)
    _assert_same(got["b"], ref_b)
