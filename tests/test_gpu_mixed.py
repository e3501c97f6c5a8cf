"""GPU parity on registers that mix qudit dimensions (section "Code style":
Circuit(dim=[2,3,4])) against the oracle: every gate kind on every target and
ordered pair, random 200-gate circuits (immediate and program), the
reductions and qf_measure, the adjoint gradient, the paper's example circuit,
and the argument checks specific to mixed dimensions."""
import itertools
import math

import numpy as np
import pytest

from gpu_util import download, gpu_lib, tol
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIMS = [[2, 3, 4, 5, 3, 2], [5, 2, 3, 4], [3, 5, 2, 4, 3, 5, 2, 3], [4, 4, 2, 2, 3]]


def upload_dims(qf, psi, dims, dtype):
    import torch
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    t = torch.from_numpy(np.ascontiguousarray(psi)).to(device="cuda", dtype=tdt)
    return qf.State(dims, len(dims), dtype, tensor=t)


def gate_list(dims, rng):
    n = len(dims)
    ops = []
    for q in range(n):
        d = dims[q]
        ops += [W.Op("h", (q,)), W.Op("x", (q,), power=d - 1), W.Op("z", (q,), power=1),
                W.Op("rot", (q,), j=0, k=d - 1, axis="x", theta=0.7),
                W.Op("rot", (q,), j=0, k=1, axis="y", theta=-1.3),
                W.Op("rot", (q,), j=d - 2, k=d - 1, axis="z", theta=2.1),
                W.Op("rot", (q,), j=d - 1, axis="g", theta=0.9),
                W.Op("u", (q,), matrix=W.haar_unitary(d, rng))]
    for c, t in itertools.permutations(range(n), 2):
        dt = dims[t]
        ops += [W.Op("sum", (c, t)),
                W.Op("crot", (c, t), j=0, k=dt - 1, axis="x", theta=0.4),
                W.Op("crot", (c, t), j=0, k=1, axis="y", theta=1.1),
                W.Op("crot", (c, t), j=0, k=1, axis="z", theta=0.3),
                W.Op("crot", (c, t), j=dt - 1, axis="g", theta=-0.6)]
        if dims[c] * dt <= 64:
            ops.append(W.Op("u", (c, t), matrix=W.haar_unitary(dims[c] * dt, rng)))
        if dims[c] == dt:
            ops.append(W.Op("swap", (c, t)))
    return ops


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims", DIMS)
def test_every_gate_every_target(orc, dims, dtype):
    qf = gpu_lib()
    n = len(dims)
    psi0 = W.uniform_state(dims, n, seed=7)
    ref0 = psi0.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi0
    st = upload_dims(qf, psi0, dims, dtype)
    for op in gate_list(dims, np.random.default_rng(sum(dims))):
        st.tensor.copy_(st.tensor.new_tensor(psi0))
        qf.apply_ops(st.handle, [op])
        got = download(st)
        want = orc.run([op], dims, n, psi=ref0)
        assert np.abs(got - want).max() <= tol(dtype), op
    st.free()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims", [[2, 3, 4, 5, 3, 2, 4], [3, 2, 5, 4, 3, 2, 3, 2, 4, 3]])
def test_random_circuit_program_and_immediate(orc, dims, dtype):
    qf = gpu_lib()
    n = len(dims)
    ops = W.mixed_random_circuit(dims, 200)
    want = orc.run(ops, dims, n)
    st = qf.State(dims, n, dtype).set_basis(0)
    qf.apply_ops(st.handle, ops)
    assert np.abs(download(st) - want).max() <= tol(dtype, 200)
    p = qf.program_from_ops(dims, n, ops)
    assert qf.qf_program_plan(p)[0] == len(ops)
    st.set_basis(0)
    qf.qf_program_run(p, st.handle)
    got = download(st)
    assert np.abs(got - want).max() <= tol(dtype, 200)
    e = qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL)
    np.testing.assert_allclose(e[:n], orc.expect_number(want, dims, n), atol=1e-11 if dtype == "c128" else 2e-5)
    assert abs(e[n] - 1) < (1e-12 if dtype == "c128" else 1e-5)
    qf.qf_program_free(p)
    st.free()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims", [[2, 3, 4], [5, 5, 5, 3, 2, 2], [3, 2, 5, 4, 3, 2, 3, 2, 4, 3, 5, 2],
                                  [7, 3, 11, 2, 13]])
def test_reductions_and_measure(orc, dims, dtype):
    """Row / column reduction of <N_q> (rows of up to 512 amplitudes, ragged
    lane tails), marginals of qudit subsets, Hermitian observables, shots."""
    qf = gpu_lib()
    n = len(dims)
    psi = W.uniform_state(dims, n, seed=11)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi
    st = upload_dims(qf, psi, dims, dtype)
    at = 1e-12 if dtype == "c128" else 1e-6
    e = qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL)
    np.testing.assert_allclose(e[:n], orc.expect_number(ref, dims, n), atol=at * max(dims))
    assert abs(qf.qf_expect(st.handle, qf.QF_OBS_NORM)[0] - orc.norm2(ref)) < at
    for q in (0, n - 1, n // 2):
        m = qf.qf_expect(st.handle, qf.QF_OBS_MARGINAL, q=q)
        np.testing.assert_allclose(m, orc.marginal(ref, dims, n, [q]), atol=at)
        O = W.haar_unitary(dims[q], np.random.default_rng(q))
        O = O + O.conj().T
        h = qf.qf_expect(st.handle, qf.QF_OBS_HERMITIAN, q=q, matrix=O)
        w = orc.expect_obs(ref, dims, n, q, O)
        assert abs(h[0] - w.real) < 10 * at and abs(h[1]) < 10 * at
    u = np.random.default_rng(5).random(20000)
    for idx in ([0], [n - 1, 0], [1, n - 1]):
        hist, probs = qf.qf_measure(st.handle, idx, shots=len(u), uniforms=u)
        np.testing.assert_allclose(probs, orc.marginal(ref, dims, n, idx), atol=at)
        assert np.array_equal(hist, orc.sample(probs, u))
    st.free()


def test_large_register_sampled(orc):
    """1.7 M amplitudes (dims 2,3,4,5 three times): 60 random gates, c64,
    every amplitude against the oracle."""
    qf = gpu_lib()
    dims = [2, 3, 4, 5] * 3
    n = len(dims)
    ops = W.mixed_random_circuit(dims, 60, seed=99)
    want = orc.run(ops, dims, n)
    st = qf.State(dims, n, "c64").set_basis(0)
    p = qf.program_from_ops(dims, n, ops)
    qf.qf_program_run(p, st.handle)
    assert np.abs(download(st) - want).max() <= 1e-5
    e = qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL)
    np.testing.assert_allclose(e[:n], orc.expect_number(want, dims, n), atol=5e-5)
    qf.qf_program_free(p)
    st.free()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("dims", [[2, 3, 4], [3, 5, 2, 4], [5, 2, 3, 2, 4, 3]])
def test_adjoint_gradient(orc, dims, dtype):
    qf = gpu_lib()
    n = len(dims)
    ops, P = W.mixed_ansatz(dims, 2)
    # a parameter shared by two gates, and a fixed-angle rotation between them
    ops = ops + [W.Op("rot", (n - 1,), j=0, k=1, axis="y", theta=0.3), W.Op("rot", (n - 1,), j=0, k=1, axis="y", param=0)]
    theta = W.normal_angles(P, seed=len(dims))
    w = np.linspace(0.5, 1.5, n)
    p = qf.program_from_ops(dims, n, ops)
    psi = qf.State(dims, n, dtype).set_basis(0)
    lam = qf.State(dims, n, dtype)
    loss, g = qf.qf_program_gradient(p, psi.handle, lam.handle, theta, w)
    want = orc.grad_bruteforce(ops, dims, n, theta, w)
    wl = orc.loss(orc.run(ops, dims, n, params=theta), dims, n, w)
    if dtype == "c128":
        assert abs(loss - wl) < 1e-12
        assert np.abs(g - want).max() < 1e-10
    else:
        assert abs(loss - wl) < 1e-5
        assert np.abs(g - want).max() < 1e-4 * max(1.0, np.abs(want).max())
    qf.qf_program_free(p)
    psi.free()
    lam.free()


def test_adjoint_with_group_gates(orc):
    """Reverse sweep through SWAP and two-qudit dense gates (group kernel on
    psi and lambda) between parametrised gates."""
    qf = gpu_lib()
    dims = [3, 2, 3, 4]
    n = 4
    rng = np.random.default_rng(4)
    ops = [W.Op("h", (q,)) for q in range(n)]
    ops += [W.Op("rot", (0,), j=0, k=2, axis="x", param=0), W.Op("swap", (0, 2)),
            W.Op("u", (1, 3), matrix=W.haar_unitary(8, rng)), W.Op("crot", (3, 2), j=1, k=2, axis="y", param=1),
            W.Op("rot", (2,), j=2, axis="g", param=2), W.Op("u", (2, 0, 1), matrix=W.haar_unitary(18, rng)),
            W.Op("crot", (1, 3), j=0, k=3, axis="z", param=0)]
    theta = np.array([0.7, -1.2, 2.0])
    w = [1.0, 2.0, 0.5, -1.0]
    p = qf.program_from_ops(dims, n, ops)
    psi = qf.State(dims, n, "c128").set_basis(0)
    lam = qf.State(dims, n, "c128")
    loss, g = qf.qf_program_gradient(p, psi.handle, lam.handle, theta, w)
    assert np.abs(g - orc.grad_bruteforce(ops, dims, n, theta, w)).max() < 1e-10
    qf.qf_program_free(p)
    psi.free()
    lam.free()


def test_code_style_example(orc):
    """dims [2, 3, 4] from |0, 1, 3>: Fourier on all, RX(pi/2) on qudit 0,
    CNOT(0, 2): every basis state has probability 1/24."""
    qf = gpu_lib()
    dims = [2, 3, 4]
    st = qf.State(dims, 3, "c128").set_basis(int(np.ravel_multi_index([0, 1, 3], dims)))
    for q in range(3):
        qf.qf_apply_h(st.handle, q)
    qf.qf_apply_rot(st.handle, 0, 0, 1, math.pi / 2, "x")
    qf.qf_apply_sum(st.handle, 0, 2)
    hist, probs = qf.qf_measure(st.handle, [0, 1], shots=600, seed=2)
    assert np.abs(probs - 1 / 6).max() < 1e-14
    assert np.abs(np.abs(download(st)) ** 2 - 1 / 24).max() < 1e-14
    assert hist.sum() == 600
    st.free()


def test_mixed_argument_checks():
    qf = gpu_lib()
    dims = [2, 3, 4]
    st = qf.State(dims, 3, "c64").set_basis(0)
    assert qf.qf_state_info(st.handle)[0] == 0 and qf.qf_state_dims(st.handle) == dims
    bad = [lambda: qf.qf_apply_swap(st.handle, 0, 1),                 # unequal dims
           lambda: qf.qf_apply_rot(st.handle, 0, 0, 2, 0.1, "x"),      # level 2 on a qubit
           lambda: qf.qf_apply_rot(st.handle, 1, 2, 0, 0.1, "g"),      # Gell-Mann index 2 < 3 is fine...
           lambda: qf.qf_apply_crot(st.handle, 2, 0, 0, 3, 0.1, "y"),  # target qubit has no level 3
           lambda: qf.qf_apply_gate(st.handle, [0, 1], np.eye(4))]     # 6 x 6 expected
    for i, f in enumerate(bad):
        if i == 2:
            f()   # valid: S_z^2 on a qutrit
            continue
        with pytest.raises(qf.QFError) as ei:
            f()
        assert ei.value.status == qf.QF_ERR_ARG
    p = qf.qf_program_create_dims(dims)
    b = qf.qf_batch_create(qf.QF_C64)
    with pytest.raises(qf.QFError) as ei:
        qf.qf_batch_add(b, p, [1.0, 0.0, 0.0])
    assert ei.value.status == qf.QF_ERR_UNSUPPORTED
    qf.qf_batch_free(b)
    qf.qf_program_free(p)
    # equal dims make an ordinary register
    u = qf.State([3, 3, 3], 3, "c64").set_basis(0)
    assert qf.qf_state_info(u.handle)[0] == 3
    u.free()
    st.free()
