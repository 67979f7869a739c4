"""The learned warm start end to end on the GPU: targets from cold FullADMM solves (first outer
step) of seeded quadcopter instances (T = 100, 1-15 obstacles), training of the network by the
library's own kernels, then cold vs warm-started solves of held-out instances.  Shows what the
network gains over the method without it: more instances converge within the budget and fewer
iterations are needed on the instances that converge either way."""
import numpy as np
import pytest

from paper_2603_02642_b300 import nrto, warmstart as WS, workloads as W

pytestmark = pytest.mark.gpu

OPTS = dict(rho=10.0, max_inner=5000, eps_p=1e-4, eps_d=1e-4, check=1, adapt_every=25)


def _solve(insts, ws=None):
    prob = nrto.Problem(insts, nrto.PREC_MIXED)
    prob.linearize()
    prob.set_trust_radius(2.0)
    if ws is not None:
        ws.apply(prob, insts)
    # Fallback trigger for the warm start: r_p above its tolerance and down by less than 1% over
    # 1000 iterations (these solves converge slowly, so a shorter window misreads slow progress).
    out = prob.solve_socp(nrto.Options(stall_every=1000 if ws else 0, stall_ratio=0.99, warm_fallback=1, **OPTS))
    fb = np.array([prob.export(nrto.F_STATS, i)[6] for i in range(len(insts))])
    return prob, out, fb


def test_learned_warm_start_gains_over_cold_start():
    train = [W.warmstart_quad(s) for s in range(1024)]
    prob, out, _ = _solve(train)
    X, Y, Mk = WS.collect_targets(prob, train, out["status"])
    prob.close()
    assert X.shape[0] > 700                      # most first-step solves converge cold
    ws = WS.WarmStart(max_batch=1024)
    hist = ws.fit(X, Y, Mk, steps=1500, batch=256, lr=1e-3)
    assert hist[-1] < 0.05 * hist[0]
    test = [W.warmstart_quad(1_000_000 + s) for s in range(256)]
    pc, oc, _ = _solve(test)
    pw, ow, fb = _solve(test, ws)
    pc.close()
    pw.close()
    conv_c, conv_w = oc["status"] == 1, ow["status"] == 1
    both = conv_c & conv_w
    ratio = ow["iters"][both].mean() / oc["iters"][both].mean()
    print(f"cold converged {conv_c.sum()}, warm converged {conv_w.sum()}, mean iteration ratio {ratio:.3f}, "
          f"fallbacks {int(fb.sum())}")
    assert conv_w.sum() >= conv_c.sum()
    assert ratio < 0.9
    ws.net.close()


def test_device_warm_start_equals_host_path():
    """nrto_set_warm_start_from_network installs exactly what predict + nrto_set_warm_start does."""
    insts = [W.warmstart_quad(3_000_000 + s) for s in range(16)]
    ws = WS.WarmStart(max_batch=64, seed=4)
    ws.deployed = True          # untrained network: the mapping, not the values, is under test
    outs = []
    for apply in (ws.apply, ws.apply_host):
        prob = nrto.Problem(insts, nrto.PREC_FP64)
        prob.linearize()
        apply(prob, insts)
        prob.solve_socp(nrto.Options(rho=10.0, max_inner=1, check=0))
        outs.append([(prob.export(nrto.F_K, i), prob.export(nrto.F_LAMP, i)) for i in range(len(insts))])
        prob.close()
    for (ka, la), (kb, lb) in zip(*outs):
        assert np.array_equal(ka, kb) and np.array_equal(la, lb)
    ws.net.close()
