"""GPU parity of whole circuits and of the reductions, through the C ABI.

* The layered Fourier / RX RY RZ / SUM-chain circuit on six qutrits in
  complex128: amplitudes and <N_q> within 1e-12 of the oracle.
* Random 200-gate sequences (Haar U, level-pair rotations, clock Z, shift X,
  SUM or controlled-RY) at d = 2..5, applied three ways -- immediate calls, a
  program with fusion off, a fused program -- within 1e-12 (complex128) and
  1e-5 (complex64) of the oracle.
* <N_q>, norm, marginals and Hermitian single-qudit observables against the
  oracle, on the chunked and the generic reduction paths.
* Closed forms on the GPU: GHZ amplitudes 1/sqrt(d), Grover P(|22>).
"""
import math

import numpy as np
import pytest

from gpu_util import download, gpu_lib, tol, upload
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_layered_circuit_c128(orc):
    qf = gpu_lib()
    d, n = 3, 6
    ops = W.layered_circuit(d, n, layers=20)
    assert len(ops) == 940
    want = orc.run(ops, d, n)
    want_e = orc.expect_number(want, d, n)
    for mode in ("immediate", "unfused", "fused"):
        st = qf.State(d, n, "c128").set_basis(0)
        if mode == "immediate":
            qf.apply_ops(st.handle, ops)
        else:
            p = qf.program_from_ops(d, n, ops, fuse=mode == "fused")
            qf.qf_program_run(p, st.handle)
            qf.qf_program_free(p)
        got = download(st)
        assert np.abs(got - want).max() <= 1e-12, mode
        e = st.expect_number()
        assert np.abs(e[:n] - want_e).max() <= 1e-12
        assert abs(e[n] - 1) <= 1e-12
        st.free()


RANDOM_SIZES = [(2, 16), (3, 10), (4, 8), (5, 7)]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("d,n", RANDOM_SIZES)
def test_random_200_gate_sequence(orc, d, n, dtype):
    qf = gpu_lib()
    ops = W.random_circuit(d, n, 200)
    psi0 = W.uniform_state(d, n, seed=11)
    want = orc.run(ops, d, n, psi0)
    for mode in ("immediate", "unfused", "fused"):
        st = upload(qf, psi0, d, n, dtype)
        if mode == "immediate":
            qf.apply_ops(st.handle, ops)
        else:
            p = qf.program_from_ops(d, n, ops, fuse=mode == "fused")
            qf.qf_program_run(p, st.handle)
            if mode == "fused":
                assert qf.qf_program_last_passes(p) < 120
            qf.qf_program_free(p)
        got = download(st)
        err = np.abs(got - want).max()
        assert err <= tol(dtype, 200), "%s %s d=%d n=%d err %.3g" % (mode, dtype, d, n, err)
        st.free()


def test_program_rerun_with_new_parameters(orc):
    qf = gpu_lib()
    d, n = 3, 8
    ops, P = W.variational_ansatz(d, n, 3)
    ops = [W.Op("h", (q,)) for q in range(n)] + ops
    p = qf.program_from_ops(d, n, ops)
    for seed in range(3):
        theta = W.normal_angles(P, seed=seed)
        st = qf.State(d, n, "c128").set_basis(0)
        qf.qf_program_run(p, st.handle, theta)
        want = orc.run(ops, d, n, params=theta)
        assert np.abs(download(st) - want).max() <= 1e-12
        st.free()
    qf.qf_program_free(p)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("d,n", [(2, 14), (2, 5), (3, 9), (3, 4), (4, 7), (5, 6), (6, 5), (7, 4), (8, 4), (9, 4), (16, 3)])
def test_reductions(orc, d, n, dtype):
    qf = gpu_lib()
    psi = W.uniform_state(d, n, seed=21)
    st = upload(qf, psi, d, n, dtype)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi
    a = 1e-12 if dtype == "c128" else 1e-6
    e = qf.qf_expect(st.handle, qf.QF_OBS_NUMBER_ALL)
    np.testing.assert_allclose(e[:n], orc.expect_number(ref, d, n), atol=a * n * d)
    assert abs(e[n] - orc.norm2(ref)) <= a
    assert abs(qf.qf_expect(st.handle, qf.QF_OBS_NORM)[0] - orc.norm2(ref)) <= a
    rng = np.random.default_rng(2)
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    O = A + A.conj().T
    for q in sorted({0, n // 2, n - 1}):
        m = qf.qf_expect(st.handle, qf.QF_OBS_MARGINAL, q=q)
        np.testing.assert_allclose(m, orc.marginal(ref, d, n, [q]), atol=a)
        h = qf.qf_expect(st.handle, qf.QF_OBS_HERMITIAN, q=q, matrix=O)
        want = orc.expect_obs(ref, d, n, q, O)
        assert abs(h[0] - want.real) <= a * 10 * d and abs(h[1]) <= a * 10 * d
    st.free()


@pytest.mark.parametrize("d,n", [(2, 12), (3, 8), (5, 5)])
def test_ghz_and_uniform_on_gpu(orc, d, n):
    qf = gpu_lib()
    st = qf.State(d, n, "c128").set_basis(0)
    qf.qf_apply_h(st.handle, 0)
    for q in range(n - 1):
        qf.qf_apply_sum(st.handle, q, q + 1)
    got = download(st)
    rep = (d ** n - 1) // (d - 1)
    want = np.zeros(d ** n, dtype=complex)
    want[[m * rep for m in range(d)]] = 1 / math.sqrt(d)
    assert np.abs(got - want).max() <= 1e-15
    np.testing.assert_allclose(st.expect_number()[:n], np.full(n, (d - 1) / 2), atol=1e-13)
    st.set_basis(0)
    for q in range(n):
        qf.qf_apply_h(st.handle, q)
    assert np.abs(download(st) - d ** (-n / 2)).max() <= 1e-14
    st.free()


def test_grover_on_gpu(orc):
    qf = gpu_lib()
    d, n = 3, 2
    st = qf.State(d, n, "c128").set_basis(0)
    qf.qf_apply_h(st.handle, 0)
    qf.qf_apply_h(st.handle, 1)
    s = download(st)
    marked = np.zeros(9, dtype=complex)
    marked[8] = 1
    qf.qf_apply_gate(st.handle, [0, 1], np.eye(9) - 2 * np.outer(marked, marked))
    qf.qf_apply_gate(st.handle, [0, 1], 2 * np.outer(s, s.conj()) - np.eye(9))
    m = qf.qf_expect(st.handle, qf.QF_OBS_MARGINAL, q=0)
    p = np.abs(download(st)) ** 2
    assert abs(p[8] - math.sin(3 * math.asin(1 / 3)) ** 2) <= 1e-14
    assert abs(m.sum() - 1) <= 1e-14
    st.free()
