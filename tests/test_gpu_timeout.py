"""Failure detection without a GPU fault: the tensor-core kernel's bounded
waits.  A diagnostic entry suppresses the signal one of the kernel's waits
depends on and limits every wait to a few milliseconds; the kernel must give
up on its own, report SHG_FLAG_TIMEOUT through the device status word and
leave the context usable (a normal projection right after is exact to the
usual tolerance)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import shgemm as OS
from synth import omega_f16, uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def test_bounded_wait_times_out_and_context_survives(shg):
    from paper_2304_04612_gb300 import _lib
    lib = _lib.load()
    m, n, k = 640, 512, 64
    A_h = uniform(m, n, seed=31)
    Om_h = omega_f16(n, k, seed=32)
    A = torch.from_numpy(A_h).cuda()
    Om = torch.from_numpy(Om_h).cuda()
    Y = torch.empty(m, k, device="cuda")
    flags = shg.new_flags()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.shg_diag_wait_timeout(m, n, k, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(Om.data_ptr()), k,
                                   ctypes.c_void_p(Y.data_ptr()), k, 5_000_000, ctypes.c_void_p(flags.data_ptr()),
                                   stream)
    assert rc == 0
    torch.cuda.synchronize()
    f = int(flags.item())
    assert f & 4, f                                   # SHG_FLAG_TIMEOUT
    assert lib.shg_flags_status(f) == 6                # SHG_ERR_TIMEOUT
    # the context is still usable: a normal projection on the same stream
    flags.zero_()
    Y2 = shg.shgemm_project(A, Om, flags=flags)
    ref = OS.project_exact(A_h, Om_h)
    err = np.linalg.norm(Y2.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    # out-of-range limits are rejected on the host
    assert lib.shg_diag_wait_timeout(m, n, k, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(Om.data_ptr()), k,
                                     ctypes.c_void_p(Y.data_ptr()), k, 10, ctypes.c_void_p(flags.data_ptr()),
                                     stream) == 1
