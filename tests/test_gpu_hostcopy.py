"""Host buffers <-> state amplitudes through the C ABI (qf_state_upload /
qf_state_download): full and partial ranges from page-locked (torch and the
library's qf_host_alloc) and pageable memory in both dtypes, a program run
between them checked against the oracle, and out-of-range or NULL arguments
rejected with QF_ERR_ARG."""
import numpy as np
import pytest

from gpu_util import gpu_lib
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,pinned", [("c64", True), ("c128", True), ("c128", False)])
def test_upload_run_download(orc, dtype, pinned):
    import torch
    qf = gpu_lib()
    d, n = 3, 9
    N = d ** n
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    psi0 = W.uniform_state(d, n, seed=4)
    h_in = torch.from_numpy(psi0).to(tdt)
    h_out = torch.zeros(N, dtype=tdt)
    if pinned:
        h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
    st = qf.State(d, n, dtype)
    qf.qf_state_upload(st.handle, h_in.data_ptr(), 0, N)
    ops = W.random_circuit(d, n, 40, seed=9)
    p = qf.program_from_ops(d, n, ops)
    qf.qf_program_run(p, st.handle)
    qf.qf_state_download(st.handle, h_out.data_ptr(), 0, N)
    torch.cuda.synchronize()
    want = orc.run(ops, d, n, psi0)
    tol = 1e-12 if dtype == "c128" else 1e-6
    assert np.abs(h_out.numpy().astype(np.complex128) - want).max() <= tol
    # partial ranges: a middle slice back and forth
    first, count = 1000, 3000
    part = torch.zeros(count, dtype=tdt)
    qf.qf_state_download(st.handle, part.data_ptr(), first, count)
    torch.cuda.synchronize()
    assert np.array_equal(part.numpy(), h_out.numpy()[first:first + count])
    part.zero_()
    qf.qf_state_upload(st.handle, part.data_ptr(), first, count)
    qf.qf_state_download(st.handle, h_out.data_ptr(), 0, N)
    torch.cuda.synchronize()
    out = h_out.numpy()
    assert np.all(out[first:first + count] == 0) and np.abs(out[:first] - want[:first]).max() <= tol
    qf.qf_program_free(p)
    st.free()


def test_bad_ranges_rejected():
    import torch
    qf = gpu_lib()
    d, n = 2, 6
    st = qf.State(d, n, "c64").set_basis(0)
    h = torch.zeros(2 ** n, dtype=torch.complex64)
    for first, count in [(-1, 4), (0, 65), (60, 5), (65, 0)]:
        with pytest.raises(qf.QFError) as ei:
            qf.qf_state_upload(st.handle, h.data_ptr(), first, count)
        assert ei.value.status == qf.QF_ERR_ARG
    with pytest.raises(qf.QFError) as ei:
        qf.qf_state_download(st.handle, 0, 0, 4)
    assert ei.value.status == qf.QF_ERR_ARG
    qf.qf_state_download(st.handle, h.data_ptr(), 64, 0)   # empty range at the end: allowed
    st.free()


def test_library_host_memory(orc):
    import torch
    qf = gpu_lib()
    d, n = 5, 6
    N = d ** n
    psi0 = W.uniform_state(d, n, seed=5)
    pin = qf.qf_host_alloc(N * 16)
    pout = qf.qf_host_alloc(N * 16)
    a_in = qf.host_array(pin, N, np.complex128)
    a_out = qf.host_array(pout, N, np.complex128)
    a_in[:] = psi0
    st = qf.State(d, n, "c128")
    qf.qf_state_upload(st.handle, pin, 0, N)
    ops = W.random_circuit(d, n, 30, seed=2)
    p = qf.program_from_ops(d, n, ops)
    qf.qf_program_run(p, st.handle)
    qf.qf_state_download(st.handle, pout, 0, N)
    torch.cuda.synchronize()
    assert np.abs(a_out - orc.run(ops, d, n, psi0)).max() <= 1e-12
    del a_in, a_out
    qf.qf_host_free(pin)
    qf.qf_host_free(pout)
    with pytest.raises(qf.QFError) as ei:
        qf.qf_host_free(pin)          # already freed
    assert ei.value.status == qf.QF_ERR_ARG
    qf.qf_program_free(p)
    st.free()
