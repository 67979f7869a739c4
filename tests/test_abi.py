"""CPU checks of the C ABI: the library builds, loads, exports every symbol include/nrto.h
declares, and rejects bad input on the host before touching a device."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2603_02642_b300 import build, nrto, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = ""
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt += open(os.path.join(ROOT, "include", f)).read()
    return sorted(set(re.findall(r"\b(nrto_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_all_declared_symbols():
    path = build.build()
    syms = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    names = {l.split()[-1] for l in syms.splitlines() if l.strip()}
    missing = [s for s in _declared() if s not in names]
    assert not missing, missing
    lib = nrto.load()
    for s in _declared():
        assert hasattr(lib, s)


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_invalid_descriptors_rejected_on_host():
    build.build()
    inst = W.unicycle(0, T=5)
    inst.nx = 4                               # wrong state dimension for the model
    with pytest.raises(nrto.NrtoError) as e:
        nrto.Problem([inst])
    assert e.value.code == 1
    inst = W.unicycle(0, T=5)
    inst.u_init[2, 0] = np.nan                # non-finite input
    with pytest.raises(nrto.NrtoError) as e:
        nrto.Problem([inst])
    assert e.value.code == 4
    inst = W.quadcopter(0, T=5, n_obs=1)
    inst.Sigma[3] = -inst.Sigma[3]            # covariance block not positive semidefinite
    with pytest.raises(nrto.NrtoError) as e:
        nrto.Problem([inst])
    assert e.value.code == 1 and b"positive semidefinite" in nrto.load().nrto_last_error()
    inst = W.unicycle(0, T=300)               # horizon beyond the model's limit
    with pytest.raises(nrto.NrtoError):
        nrto.Problem([inst])
    with pytest.raises(nrto.NrtoError) as e:   # an empty batch
        nrto.Problem([])
    assert e.value.code == 1


@pytest.mark.skipif(_has_gpu(), reason="checks the no-device error path")
def test_create_without_device_reports_cuda_error():
    build.build()
    with pytest.raises(nrto.NrtoError) as e:
        nrto.Problem([W.unicycle(0, T=5)])
    assert e.value.code == 2


@pytest.mark.skipif(_has_gpu(), reason="checks validation on the host before the device is used")
def test_singular_sigma_blocks_pass_validation():
    """A disturbance map Γ_i of lower rank gives Σ_i = Γ_i S_i^{-1} Γ_iᵀ singular: validation accepts it
    (creation then stops at the missing device, not at the descriptor check)."""
    build.build()
    inst = W.unicycle(0, T=5)
    inst.Sigma[:, 2, 2] = 0.0
    with pytest.raises(nrto.NrtoError) as e:
        nrto.Problem([inst])
    assert e.value.code == 2
