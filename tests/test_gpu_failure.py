"""Failure handling without a GPU fault: a host-side bounded wait that
expires.

esmf_fock_build_host waits for its build with a limit; a limit far shorter
than the build makes the wait give up with ESMF_ERR_TIMEOUT while the work
keeps running on the device.  Nothing faults or hangs: once the caller has
synchronised, the same handle must build again and give the right result.
"""
import numpy as np
import pytest

from paper_2002_00322_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def relerr(x, r):
    return float(np.linalg.norm(x - r)) / max(float(np.linalg.norm(r)), 1e-300)


def test_host_entry_wait_expires_then_handle_recovers(esmf):
    import torch
    # 240-function ribbon, integral-direct FP32, 8 densities: tens of
    # milliseconds per build, far above the 1 ms limit
    w = W.direct(length=30, m=8)
    D = np.ascontiguousarray(w.D)
    with esmf.FockBuilder(w.basis, w.tol, "direct", "fp32") as fb:
        Jd, Kd, _, _ = fb.build(torch.from_numpy(D).cuda())
        torch.cuda.synchronize()
        # page-locked host buffers: copies to pageable memory would block
        # until the build is done, before the bounded wait even starts
        Dp = torch.from_numpy(D).pin_memory()
        Jp = torch.empty(D.shape, dtype=torch.float64).pin_memory()
        Kp = torch.empty(D.shape, dtype=torch.float64).pin_memory()
        with pytest.raises(esmf.EsmfError) as e:
            fb.build_host(Dp.numpy(), Jp.numpy(), Kp.numpy(), timeout_ms=1)
        assert e.value.code == esmf.ESMF_ERR_TIMEOUT
        assert "did not finish" in esmf.esmf_last_error()
        torch.cuda.synchronize()       # the timed-out build finishes on the device
        assert fb.device_error() == 0
        J, K, _ = fb.build_host(Dp.numpy(), Jp.numpy(), Kp.numpy(), timeout_ms=60000)
    for k in range(w.m):
        assert relerr(J[k], Jd[k].cpu().numpy()) <= 1e-12
        assert relerr(K[k], Kd[k].cpu().numpy()) <= 1e-12
