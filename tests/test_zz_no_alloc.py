"""ed_dot_noalloc, the reduction for callers that cannot allocate device memory (a loop
that must not stall the device, or a framework that owns all device memory), checked
through the C ABI against ed_dot on the same vectors, on two calls in a row."""
import ctypes

import numpy as np
import pytest

import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["float64", "float32", "complex128", "complex64"])
def test_dot_noalloc_matches_ed_dot(dtype):
    import paper_1804_05028_gb300 as ed
    dt = getattr(torch, dtype)
    p = w.config_chain16() if not dtype.startswith("complex") else w.chain(16, 2, k=3, n_up=8)
    B = ed.build_basis_from(p)
    states, _ = B.export()
    x = torch.from_numpy(w.state_uniform(states, 3)).cuda()
    y = torch.from_numpy(w.state_uniform(states, 4)).cuda()
    if dt.is_complex:
        x = torch.complex(x, torch.from_numpy(w.state_uniform(states, 5)).cuda())
        y = torch.complex(y, torch.from_numpy(w.state_uniform(states, 6)).cuda())
    x, y = x.to(dt), y.to(dt)
    ref = B.dot(x, y)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):                       # the fixed scratch keeps the previous call's data
        ed.dot_noalloc(x, y, out)
        torch.cuda.synchronize()
        got = complex(out[0].item(), out[1].item())
        assert abs(got - complex(ref)) <= 1e-12 * max(1.0, abs(ref))
    # a long vector spanning many blocks of the fixed partial array
    n = 3_000_001
    a = torch.rand(n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, dtype=torch.float64, device="cuda")
    ed.dot_noalloc(a, b, out)
    torch.cuda.synchronize()
    exact = float(np.dot(a.cpu().numpy(), b.cpu().numpy()))
    assert abs(out[0].item() - exact) <= 1e-12 * abs(exact)


def test_dot_noalloc_refuses_oversized_input():
    import paper_1804_05028_gb300 as ed
    L = ed.lib()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = L.ed_dot_noalloc(None, None, (1 << 30) + 1, ed.F64, ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1 and b"2^30" in L.ed_last_error()
