"""shg_cholqr2_static, the CholeskyQR2 entry point that allocates nothing,
against the workspace entry point shg_cholqr2 on the same inputs.

Collected last on purpose: it must also pass after every other test has run
in the same process (device memory already handed out by the caching
allocator, the library's other kernels already loaded)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call_static(lib, X, flags):
    fl = ctypes.c_void_p(flags.data_ptr()) if flags is not None else ctypes.c_void_p(0)
    return lib.shg_cholqr2_static(X.shape[0], X.shape[1], ctypes.c_void_p(X.data_ptr()), X.stride(0), fl,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("m,k", [(4099, 48), (1024, 64), (300, 9)])
def test_static_matches_workspace_entry_twice(m, k):
    import paper_2304_04612_gb300 as shg
    from paper_2304_04612_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(1000 + m + k)
    X0 = torch.from_numpy(rng.standard_normal((m, k)).astype(np.float32)).to(dev)
    ref = shg.shg_cholqr2(X0.clone())
    torch.cuda.synchronize()
    for call in range(2):
        X = X0.clone()
        flags = shg.new_flags(dev)
        assert _call_static(lib, X, flags) == 0
        torch.cuda.synchronize()
        assert int(flags.item()) == 0, f"call {call}: device flags {int(flags.item())}"
        # same launches on the same inputs: equal up to FP32 rounding
        err = (X - ref).abs().max().item()
        assert err <= 1e-6, f"call {call}: max |Q_static - Q_workspace| = {err}"


def test_static_null_flags_and_size_limit():
    import paper_2304_04612_gb300 as shg
    from paper_2304_04612_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(7)
    X0 = torch.from_numpy(rng.standard_normal((2048, 32)).astype(np.float32)).to(dev)
    ref = shg.shg_cholqr2(X0.clone())
    X = X0.clone()
    assert _call_static(lib, X, None) == 0
    torch.cuda.synchronize()
    assert (X - ref).abs().max().item() <= 1e-6
    # beyond the 32 MiB static scratch: rejected on the host, before any launch
    big = torch.empty(1, dtype=torch.float32, device=dev)
    rc = lib.shg_cholqr2_static(1 << 20, 64, ctypes.c_void_p(big.data_ptr()), 64, ctypes.c_void_p(0),
                                ctypes.c_void_p(0))
    assert rc == 4  # SHG_ERR_WORKSPACE


def test_static_allocates_nothing():
    """Observed, not only read: the device's free memory is the same before
    and after a call that follows the first one on the device, and the
    result equals the workspace entry point's."""
    import paper_2304_04612_gb300 as shg
    from paper_2304_04612_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(11)
    X0 = torch.from_numpy(rng.standard_normal((3000, 40)).astype(np.float32)).to(dev)
    ref = shg.shg_cholqr2(X0.clone())
    flags = shg.new_flags(dev)
    X = X0.clone()
    assert _call_static(lib, X, flags) == 0  # first call: the scratch's address is looked up once
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    X.copy_(X0)
    assert _call_static(lib, X, flags) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert int(flags.item()) == 0
    assert (X - ref).abs().max().item() <= 1e-6
