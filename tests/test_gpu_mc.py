"""GPU parity of the multi-controlled gates (the paper's Toffoli and
multi-controlled NOT, read as target += shift * product of control levels, and
the level-controlled single-qudit gate) against the oracle: immediate calls
on uniform and mixed registers, fused programs with such gates between tile
passes, and adjoint gradients that sweep back through them."""
import numpy as np
import pytest

from gpu_util import download, gpu_lib, tol, upload
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def mc_ops(dims, rng):
    n = len(dims)
    V = lambda q: W.haar_unitary(dims[q], rng)
    return [W.Op("mcx", (0, n - 1), power=1), W.Op("mcx", (n - 1, 1, 0), power=1),
            W.Op("mcx", (1, 3, 2), power=2), W.Op("mcx", (n - 2, 0, 1, n - 1), power=1),
            W.Op("mcu", (2, 0), levels=(1,), matrix=V(0)),
            W.Op("mcu", (0, n - 1, 1), levels=(dims[0] - 1, 0), matrix=V(1)),
            W.Op("mcu", (3, 1, 0, 2, n - 1), levels=(1, 1, 1, 0), matrix=V(n - 1))]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims", [[3] * 6, [2] * 10, [4] * 5, [2, 3, 4, 3, 2], [5, 2, 3, 2, 4, 3]])
def test_mc_gates_immediate(orc, dims, dtype):
    qf = gpu_lib()
    n = len(dims)
    psi0 = W.uniform_state(dims, n, seed=3)
    ref0 = psi0.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi0
    import torch
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    st = qf.State(dims, n, dtype, tensor=torch.from_numpy(psi0).to("cuda", tdt))
    for op in mc_ops(dims, np.random.default_rng(n)):
        st.tensor.copy_(st.tensor.new_tensor(psi0))
        qf.apply_ops(st.handle, [op])
        want = orc.run([op], dims, n, psi=ref0)
        assert np.abs(download(st) - want).max() <= tol(dtype), op
    st.free()


def test_qubit_toffoli_basis_states():
    qf = gpu_lib()
    for idx in range(8):
        st = qf.State(2, 3, "c128").set_basis(idx)
        qf.qf_apply_mcx(st.handle, [0, 1], 2)
        got = int(np.argmax(np.abs(download(st))))
        assert got == (idx ^ 1 if idx >= 6 else idx)
        st.free()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("d,n", [(3, 9), (2, 14), (5, 5)])
def test_mc_gates_in_fused_program(orc, d, n, dtype):
    """Random gates with multi-controlled gates between them: the planner
    runs each MC gate as a pass of its own between tile passes."""
    qf = gpu_lib()
    rng = np.random.default_rng(d * n)
    ops = W.random_circuit(d, n, 60)
    mc = mc_ops([d] * n, rng)
    ops = ops[:15] + mc[:3] + ops[15:40] + mc[3:] + ops[40:]
    p = qf.program_from_ops(d, n, ops)
    st = qf.State(d, n, dtype).set_basis(0)
    qf.qf_program_run(p, st.handle)
    want = orc.run(ops, d, n)
    assert np.abs(download(st) - want).max() <= tol(dtype, len(ops))
    passes = qf.qf_program_plan(p)[0]
    assert passes >= len(mc) + 1
    qf.qf_program_free(p)
    st.free()


@pytest.mark.parametrize("dims", [[3] * 5, [2, 3, 4, 3]])
def test_mc_gates_in_adjoint(orc, dims):
    qf = gpu_lib()
    n = len(dims)
    ops, P = W.mixed_ansatz(dims, 2)
    rng = np.random.default_rng(1)
    mc = mc_ops(dims, rng)[:5] if n < 5 else mc_ops(dims, rng)
    ops = ops[: len(ops) // 2] + mc + ops[len(ops) // 2:]
    theta = W.normal_angles(P, seed=5)
    w = np.linspace(1.0, 2.0, n)
    p = qf.program_from_ops(dims if len(set(dims)) > 1 else dims[0], n, ops)
    psi = qf.State(dims, n, "c128").set_basis(0)
    lam = qf.State(dims, n, "c128")
    loss, g = qf.qf_program_gradient(p, psi.handle, lam.handle, theta, w)
    assert np.abs(g - orc.grad_bruteforce(ops, dims, n, theta, w)).max() < 1e-10
    assert abs(loss - orc.loss(orc.run(ops, dims, n, params=theta), dims, n, w)) < 1e-12
    qf.qf_program_free(p)
    psi.free()
    lam.free()


def test_mc_argument_checks():
    qf = gpu_lib()
    st = qf.State(3, 4, "c64").set_basis(0)
    for f in (lambda: qf.qf_apply_mcx(st.handle, [], 1),
              lambda: qf.qf_apply_mcx(st.handle, [0, 0], 1),
              lambda: qf.qf_apply_mcx(st.handle, [0, 1], 1),
              lambda: qf.qf_apply_mcu(st.handle, [0], [3], 1, np.eye(3)),
              lambda: qf.qf_apply_mcu(st.handle, [0], [1], 1, np.eye(2))):
        with pytest.raises(qf.QFError) as ei:
            f()
        assert ei.value.status == qf.QF_ERR_ARG
    p = qf.program_from_ops(3, 4, [W.Op("mcx", (0, 1, 2))])
    b = qf.qf_batch_create(qf.QF_C64)
    with pytest.raises(qf.QFError) as ei:
        qf.qf_batch_add(b, p, [1.0, 0, 0, 0])
    assert ei.value.status == qf.QF_ERR_UNSUPPORTED
    qf.qf_batch_free(b)
    qf.qf_program_free(p)
    st.free()
