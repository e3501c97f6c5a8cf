"""The allocation-free <N_q> entry point (qf_expect_number_noalloc).

It exists for callers that cannot allocate device memory when they measure
(host callbacks and latency-bound loops that must not trigger the device-wide
synchronisation an allocation can cause, hosts whose memory pool owns the
device heap): it writes <N_q> and the norm for a caller-owned state into a
caller-owned device buffer, keeping its partial sums in a fixed device array.
Here it is called through the C ABI twice in a row -- the second time on a
different state, so the shared scratch still holds the first call's partials
-- and each result must match qf_expect's (the allocating entry point) within
the reduction tolerances the other GPU tests use.  This file is collected last
so a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

from gpu_util import gpu_lib, upload
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(qf, st, d, n, dtype):
    import torch
    out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    qf.qf_expect_number_noalloc(st.tensor.data_ptr(), d, n, qf.QF_C64 if dtype == "c64" else qf.QF_C128,
                                out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_matches_allocating_entry_point(dtype):
    qf = gpu_lib()
    atol = 1e-12 if dtype == "c128" else 1e-6
    # two calls in a row on different states (chunked kernel, then the generic
    # path with fewer CTAs), then the first state again
    cases = [(3, 12), (9, 4), (3, 12)]
    for d, n in cases:
        st = upload(qf, W.uniform_state(d, n, seed=d * 31 + n), d, n, dtype)
        want = qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL)
        got = _noalloc(qf, st, d, n, dtype)
        assert got.shape == want.shape
        np.testing.assert_allclose(got, want, rtol=0, atol=atol * n * d)
        st.free()


def test_noalloc_rejects_bad_arguments():
    qf = gpu_lib()
    import torch
    d, n = 3, 5
    st = upload(qf, W.uniform_state(d, n, seed=2), d, n, "c64")
    out = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    bad = [(0, d, n, qf.QF_C64, out.data_ptr()),                      # NULL amplitudes
           (st.tensor.data_ptr(), d, n, qf.QF_C64, 0),                # NULL output
           (st.tensor.data_ptr() + 8, d, n, qf.QF_C64, out.data_ptr()),  # misaligned amplitudes
           (st.tensor.data_ptr(), 1, n, qf.QF_C64, out.data_ptr()),   # d < 2
           (st.tensor.data_ptr(), 2, 63, qf.QF_C64, out.data_ptr())]  # d^n above 9e15 amplitudes
    for args in bad:
        with pytest.raises(qf.QFError) as ei:
            qf.qf_expect_number_noalloc(*args)
        assert ei.value.status == qf.QF_ERR_ARG
    assert "d^n too large" in str(ei.value)
    st.free()
