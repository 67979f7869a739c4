"""nrto_solve through its CUDA graph: the captured launch sequence is replayed by later calls with the
same options and gives bitwise the results of direct launches; new options recapture."""
import numpy as np
import pytest
import torch

from paper_2603_02642_b300 import nrto, workloads as W

pytestmark = pytest.mark.gpu


def _batch():
    return [W.unicycle(21, T=30, n_obs=3), W.quadcopter(22, T=20, n_obs=2), W.arm(24, T=8), W.franka(3, T=10)]


def test_graph_replays_match_direct_launches():
    st = torch.cuda.Stream()
    o = nrto.Options(rho=10.0, max_inner=40, max_inner_final=120, check=1, adapt_every=10, stall_every=50,
                     carry=1)
    direct = nrto.Problem(_batch(), nrto.PREC_MIXED, stream=st.cuda_stream)
    direct.set_graph(False)
    ref = direct.solve(o, n_outer=4)
    ref_st = direct.stats()
    g = nrto.Problem(_batch(), nrto.PREC_MIXED, stream=st.cuda_stream)
    l0 = g.kernel_launches()
    outs = [g.solve(o, n_outer=4) for _ in range(3)]
    assert g.graph_info() == (1, 3)
    # each replay counts the kernels it launches, as many as one direct solve
    d0 = direct.kernel_launches()
    direct.solve(o, n_outer=4)
    assert g.kernel_launches() - l0 == 3 * (direct.kernel_launches() - d0)
    for out in outs:
        for i in range(len(ref["K"])):
            assert np.array_equal(out["K"][i], ref["K"][i]) and np.array_equal(out["u_bar"][i], ref["u_bar"][i])
        assert np.array_equal(out["merit"], ref["merit"])
    assert np.array_equal(g.stats()["cum_iters"], ref_st["cum_iters"])
    # other options: a new capture, whose results again equal the direct path's
    o2 = nrto.Options(rho=10.0, max_inner=30, check=1, carry=0)
    a = g.solve(o2, n_outer=2)
    b = direct.solve(o2, n_outer=2)
    assert g.graph_info() == (2, 4)
    for i in range(len(a["K"])):
        assert np.array_equal(a["K"][i], b["K"][i])
    g.close()
    direct.close()


def test_default_stream_problems_launch_directly():
    p = nrto.Problem(_batch()[:1], nrto.PREC_FP64)
    p.solve(nrto.Options(rho=10.0, max_inner=10, check=0), n_outer=1)
    assert p.graph_info() == (0, 0)
    p.close()
