"""Pins of the oracle's gate application and reductions (CPU only).

The oracle applies a gate by gathering each group of amplitudes it couples.
Here the same gates are applied as full d^n x d^n matrices built independently:
numpy Kronecker products I (x) .. (x) U (x) .. (x) I (qudit 0 leftmost, the
decimal representation of the Generalized CNOT gate section) for one qudit,
and digit-tuple enumeration for several qudits (the index rule of the SUM and
SWAP sections).  The reductions are checked against numpy digit arithmetic and
reshape-based marginals.
"""
import itertools

import numpy as np
import pytest

from paper_2409_17716_gb300 import workloads as W


def kron_1q(d, n, q, U):
    M = np.ones((1, 1), dtype=complex)
    for p in range(n):
        M = np.kron(M, U if p == q else np.eye(d))
    return M


def digits(i, d, n):
    return [(i // d ** (n - 1 - q)) % d for q in range(n)]


def full_kq(d, n, targets, U):
    """<i'| M |i> = U[r(i'), r(i)] if i' and i agree off the targets."""
    N = d ** n
    M = np.zeros((N, N), dtype=complex)
    k = len(targets)
    for i in range(N):
        di = digits(i, d, n)
        col = 0
        for t in targets:
            col = col * d + di[t]
        for row in range(d ** k):
            dj = list(di)
            rem = row
            for t in reversed(targets):
                dj[t] = rem % d
                rem //= d
            ip = sum(dj[q] * d ** (n - 1 - q) for q in range(n))
            M[ip, i] = U[row, col]
    return M


def rand_state(d, n, seed):
    return W.uniform_state(d, n, seed=seed)


SIZES = [(2, 1), (2, 3), (2, 4), (3, 1), (3, 2), (3, 4), (4, 3), (5, 3)]


@pytest.mark.parametrize("d,n", SIZES)
def test_single_qudit_matches_kronecker(orc, d, n):
    rng = np.random.default_rng(d * 100 + n)
    gates = [orc.fourier(d), orc.shift(d, 1), orc.clock(d, 1), W.haar_unitary(d, rng),
             orc.rot(d, 0, 1, 0.7, "x"), orc.rot(d, 0, d - 1, 1.9, "y"), orc.rot(d, 0, 1, 2.3, "z"),
             orc.rot(d, d - 1, 0, 0.4, "g")]
    for q in range(n):
        for U in gates:
            psi = rand_state(d, n, seed=q)
            want = kron_1q(d, n, q, U) @ psi
            got = orc.apply(psi.copy(), d, n, [q], U)
            np.testing.assert_allclose(got, want, atol=1e-14)


def test_kron_helper_agrees_with_enumeration():
    """The two independent full-matrix builders agree on one-qudit gates."""
    rng = np.random.default_rng(0)
    for d, n in [(2, 3), (3, 3)]:
        for q in range(n):
            U = W.haar_unitary(d, rng)
            np.testing.assert_allclose(kron_1q(d, n, q, U), full_kq(d, n, [q], U), atol=1e-15)


@pytest.mark.parametrize("d,n", [(2, 3), (3, 2), (3, 3), (4, 3), (5, 2)])
def test_two_qudit_gates_match_full_matrix(orc, d, n):
    rng = np.random.default_rng(7 * d + n)
    for c, t in itertools.permutations(range(n), 2):
        for U in [orc.sum_gate(d), orc.swap_gate(d), orc.crot(d, 0, 1, 1.1, "y"),
                  orc.crot(d, 0, d - 1, 0.6, "x"), orc.crot(d, 0, 1, 2.0, "z"),
                  W.haar_unitary(d * d, rng)]:
            psi = rand_state(d, n, seed=c * 10 + t)
            want = full_kq(d, n, [c, t], U) @ psi
            got = orc.apply(psi.copy(), d, n, [c, t], U)
            np.testing.assert_allclose(got, want, atol=1e-13)


def test_sum_index_rule_on_registers(orc):
    """SUM(c, t) maps basis |.. k_c .. k_t ..> to |.. k_c .. k_t + k_c ..>, both c < t and c > t."""
    for d, n in [(3, 3), (4, 3), (2, 4)]:
        for c, t in itertools.permutations(range(n), 2):
            for i in range(d ** n):
                dig = digits(i, d, n)
                psi = orc.basis(d, n, i)
                orc.apply(psi, d, n, [c, t], orc.sum_gate(d))
                dig[t] = (dig[t] + dig[c]) % d
                j = sum(dig[q] * d ** (n - 1 - q) for q in range(n))
                assert psi[j] == 1 and np.count_nonzero(psi) == 1


def test_three_qudit_custom_gate(orc):
    rng = np.random.default_rng(3)
    d, n = 2, 4
    for targets in [(0, 1, 2), (3, 1, 0), (2, 0, 3)]:
        U = W.haar_unitary(d ** 3, rng)
        psi = rand_state(d, n, seed=11)
        np.testing.assert_allclose(orc.apply(psi.copy(), d, n, list(targets), U),
                                   full_kq(d, n, list(targets), U) @ psi, atol=1e-13)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4), (5, 3)])
def test_reductions(orc, d, n):
    psi = rand_state(d, n, seed=5)
    p = np.abs(psi) ** 2
    assert abs(orc.norm2(psi) - p.sum()) < 1e-14
    idx = np.arange(d ** n)
    want = [float(np.sum(((idx // d ** (n - 1 - q)) % d) * p)) for q in range(n)]
    np.testing.assert_allclose(orc.expect_number(psi, d, n), want, atol=1e-14)
    T = p.reshape([d] * n)
    for sel in [(0,), (n - 1,), (0, n - 1), (n - 1, 0)]:
        other = tuple(a for a in range(n) if a not in sel)
        m = T.sum(axis=other)
        if list(sel) != sorted(sel):
            m = m.T
        np.testing.assert_allclose(orc.marginal(psi, d, n, list(sel)), m.reshape(-1), atol=1e-14)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    O = A + A.conj().T
    for q in range(n):
        want = np.vdot(psi, kron_1q(d, n, q, O) @ psi)
        got = orc.expect_obs(psi, d, n, q, O)
        assert abs(got - want) < 1e-13
    b = rand_state(d, n, seed=6)
    assert abs(orc.inner(psi, b) - np.vdot(psi, b)) < 1e-14


def test_invalid_apply(orc):
    psi = orc.basis(3, 3)
    with pytest.raises(ValueError):
        orc.apply(psi, 3, 3, [0, 0], np.eye(9))
    with pytest.raises(ValueError):
        orc.apply(psi, 3, 3, [3], np.eye(3))


def test_thread_count_does_not_change_results(orc):
    """The CPU baseline times the oracle on one thread and on all cores; the
    amplitudes must be bit-identical either way (OpenMP only splits
    independent amplitude groups)."""
    from paper_2409_17716_gb300 import workloads as W
    d, n = 3, 8
    ops = W.random_circuit(d, n, 40)
    before = orc.get_threads()
    try:
        orc.set_threads(1)
        one = orc.run(ops, d, n)
        orc.set_threads(4)
        many = orc.run(ops, d, n)
    finally:
        orc.set_threads(before)
    assert np.array_equal(one, many)
