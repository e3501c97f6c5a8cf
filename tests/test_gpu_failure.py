"""Allocation failures are error returns, not faults: a state or a batch
larger than the device's memory makes qf_state_init / qf_batch_build return
QF_ERR_OOM with a message, and the library keeps working afterwards (a small
state is created, a circuit runs and matches the oracle).  The failing
allocations are plain cudaMalloc calls that the driver refuses; nothing is
launched for them."""
import numpy as np
import pytest

from gpu_util import download, gpu_lib
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _still_works(qf, orc):
    d, n = 3, 6
    ops = W.layered_circuit(d, n, layers=1)
    st = qf.State(d, n, "c128").set_basis(0)
    p = qf.program_from_ops(d, n, ops)
    qf.qf_program_run(p, st.handle)
    assert np.abs(download(st) - orc.run(ops, d, n)).max() <= 1e-12
    qf.qf_program_free(p)
    st.free()


def test_state_init_over_capacity_returns_oom(orc):
    import torch
    qf = gpu_lib()
    _, total = torch.cuda.mem_get_info()
    # 2^50 complex128 amplitudes: 18 PB, far beyond any device
    assert 16 * 2 ** 50 > total
    with pytest.raises(qf.QFError) as ei:
        qf.qf_state_init(2, 50, qf.QF_C128)
    assert ei.value.status == qf.QF_ERR_OOM
    assert "allocation" in ei.value.message
    _still_works(qf, orc)


def test_batch_build_over_capacity_returns_oom(orc):
    import torch
    qf = gpu_lib()
    _, total = torch.cuda.mem_get_info()
    d, n, count = 3, 19, 16
    # 16 circuits of 3^19 complex128 amplitudes: each state alone is 18.6 GB,
    # together more than the device holds
    assert count * 16 * d ** n > total
    ops, P = W.variational_ansatz(d, n, 1, entangler="chain")
    b = qf.qf_batch_create(qf.QF_C128)
    progs = []
    for _ in range(count):
        p = qf.program_from_ops(d, n, ops)
        qf.qf_batch_add(b, p, [1.0] + [0.0] * (n - 1))
        progs.append(p)
    with pytest.raises(qf.QFError) as ei:
        qf.qf_batch_build(b, P)
    assert ei.value.status == qf.QF_ERR_OOM
    qf.qf_batch_free(b)
    for p in progs:
        qf.qf_program_free(p)
    torch.cuda.synchronize()
    _still_works(qf, orc)
