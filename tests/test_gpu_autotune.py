"""Launch-mapping autotuner: every mapping of the persistent launches (kinds one after another, at
the same time, with the SMs split between kinds) gives bitwise the same results, and nrto_autotune
times each on the caller's batch and keeps the fastest."""
import numpy as np
import pytest
import torch

from paper_2603_02642_b300 import nrto, workloads as W

pytestmark = pytest.mark.gpu


def test_every_launch_mapping_gives_the_same_results():
    insts = W.batched_mix(64, base_seed=777) + [W.arm(5, T=12), W.franka(2, T=10)]
    st = torch.cuda.Stream()
    o = nrto.Options(rho=10.0, max_inner=30, max_inner_final=80, check=1, adapt_every=10, stall_every=40, carry=1)
    ref = None
    for m in range(nrto.NMAPPING):
        p = nrto.Problem(insts, nrto.PREC_MIXED, stream=st.cuda_stream)
        p.set_launch_mapping(m)
        out = p.solve(o, n_outer=3)
        stats = p.stats()
        if ref is None:
            ref = (out, stats)
        else:
            for i in range(len(insts)):
                assert np.array_equal(out["K"][i], ref[0]["K"][i]) and np.array_equal(out["u_bar"][i], ref[0]["u_bar"][i])
            assert np.array_equal(stats["cum_iters"], ref[1]["cum_iters"])
        p.close()


def test_autotune_picks_the_fastest_mapping():
    insts = W.batched_mix(296, base_seed=10000)
    st = torch.cuda.Stream()
    p = nrto.Problem(insts, nrto.PREC_MIXED, stream=st.cuda_stream)
    o = nrto.Options(rho=10.0, max_inner=40, check=0)
    chosen, ms = p.autotune(o, n_outer=1, reps=2)
    assert 0 <= chosen < nrto.NMAPPING and np.all(ms > 0) and chosen == int(np.argmin(ms))
    with pytest.raises(nrto.NrtoError):
        p.set_launch_mapping(nrto.NMAPPING)
    p.close()
