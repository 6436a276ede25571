"""krs_gemv_t_noalloc: the tall-skinny product V^T u for callers that cannot allocate device
memory (a framework holding the device's memory in its own pool, a latency-bound loop that
cannot pay for an allocation, code where another component owns every allocation).  It
keeps its partial sums in a fixed array of the library instead of allocating them; here
it is checked, through the C ABI, against krs_gemv_t (which allocates) on two calls in a
row with different data (bitwise equal results: the two run the same kernels in the same
partition), so leftovers of the first call cannot leak into the second."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case(gpu_lib, n, k, seed):
    import torch
    rng = np.random.default_rng(seed)
    ld = (n + 31) // 32 * 32
    V = np.zeros((k, ld))
    V[:, :n] = rng.standard_normal((k, n))
    u = np.zeros(ld)
    u[:n] = rng.standard_normal(n)
    Vd = torch.as_tensor(V, device="cuda")
    ud = torch.as_tensor(u, device="cuda")
    t_ref = torch.zeros(k, device="cuda", dtype=torch.float64)
    t_na = torch.full((k,), np.nan, device="cuda", dtype=torch.float64)
    st = torch.cuda.current_stream().cuda_stream
    assert gpu_lib.krs_gemv_t(n, k, Vd.data_ptr(), ld, ud.data_ptr(), t_ref.data_ptr(), st) == 0
    assert gpu_lib.krs_gemv_t_noalloc(n, k, Vd.data_ptr(), ld, ud.data_ptr(), t_na.data_ptr(), st) == 0
    torch.cuda.synchronize()
    a, b = t_na.cpu().numpy(), t_ref.cpu().numpy()
    # same kernels, partition and summation order as krs_gemv_t: the same bits
    assert np.all(np.isfinite(a))
    assert np.array_equal(a, b)
    # and both within the tall-skinny kernel tests' rounding bound of the host product
    Vn = V[:, :n]
    bound = 1e-15 * np.sqrt(n) * (np.abs(Vn) @ np.abs(u[:n])) * 8 + 1e-300
    assert np.all(np.abs(a - Vn @ u[:n]) <= bound)


def test_noalloc_matches_allocating_entry_point_twice(gpu_lib):
    _case(gpu_lib, 104544, 300, 1)   # first call: sets up the scratch address on this device
    _case(gpu_lib, 20011, 37, 2)     # second call: different shape and data, same scratch


def test_noalloc_rejects_k_beyond_its_scratch(gpu_lib):
    import torch
    n, k = 1000, 1025
    V = torch.zeros(k * 1024, device="cuda", dtype=torch.float64)
    t = torch.zeros(k, device="cuda", dtype=torch.float64)
    st = torch.cuda.current_stream().cuda_stream
    assert gpu_lib.krs_gemv_t_noalloc(n, k, V.data_ptr(), 1024, V.data_ptr(), t.data_ptr(), st) == 1
    assert b"1024" in gpu_lib.krs_last_error()
