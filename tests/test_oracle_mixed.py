"""Pins of the oracle on mixed-dimension registers (section "Code style":
Circuit(dim=[2,3,4]); CPU only).

* Every gate kind on every target (and ordered pair) against the full
  operator built independently: basis states enumerated with numpy's
  ravel_multi_index / unravel_index over the register's dimensions, so no
  stride arithmetic of the oracle is reused.
* The two-qudit builders with unequal dimensions decompose into blocks of
  single-qudit gates pinned elsewhere: SUM = sum_c |c><c| (x) X_{d_t}^c and
  CR = sum_m |m><m| (x) R_{d_t}(m theta).
* Marginals and <N_q> against numpy reductions of |psi|^2 reshaped to dims.
* Closed forms: Fourier on every qudit gives the uniform state with
  <N_q> = (d_q - 1)/2; a GHZ ladder from a smallest qudit; H^2 |x> = |-x mod d_q>;
  the example circuit of the "Code style" section gives 1/24 on every basis state.
* Gradients: derivative circuits against central differences.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2409_17716_gb300 import workloads as W

DIMS = [[2, 3, 4], [3, 2, 5, 2], [4, 2, 3]]


def full_operator(U, dims, targets):
    dims = list(dims)
    N = int(np.prod(dims))
    tdims = [dims[t] for t in targets]
    F = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        dig = list(np.unravel_index(i, dims))
        col = int(np.ravel_multi_index([dig[t] for t in targets], tdims))
        for r in range(U.shape[0]):
            if U[r, col] == 0:
                continue
            new = list(dig)
            for t, v in zip(targets, np.unravel_index(r, tdims)):
                new[t] = int(v)
            F[int(np.ravel_multi_index(new, dims)), i] += U[r, col]
    return F


def rand_state(N, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("dims", DIMS)
def test_every_gate_vs_full_operator(orc, dims):
    n = len(dims)
    N = int(np.prod(dims))
    rng = np.random.default_rng(sum(dims))
    ops = []
    for q in range(n):
        d = dims[q]
        ops += [W.Op("h", (q,)), W.Op("x", (q,), power=d - 1), W.Op("z", (q,), power=1),
                W.Op("rot", (q,), j=0, k=d - 1, axis="x", theta=0.7),
                W.Op("rot", (q,), j=0, k=1, axis="y", theta=-1.3),
                W.Op("rot", (q,), j=0, k=d - 1, axis="z", theta=2.1),
                W.Op("rot", (q,), j=d - 1, axis="g", theta=0.9),
                W.Op("u", (q,), matrix=W.haar_unitary(d, rng))]
    for c, t in itertools.permutations(range(n), 2):
        dt = dims[t]
        ops += [W.Op("sum", (c, t)),
                W.Op("crot", (c, t), j=0, k=dt - 1, axis="x", theta=0.4),
                W.Op("crot", (c, t), j=0, k=1, axis="y", theta=1.1),
                W.Op("crot", (c, t), j=dt - 1, axis="g", theta=-0.6),
                W.Op("u", (c, t), matrix=W.haar_unitary(dims[c] * dt, rng))]
        if dims[c] == dt:
            ops.append(W.Op("swap", (c, t)))
    psi0 = rand_state(N, 5)
    for op in ops:
        t, U = orc.op_matrix(op, dims)
        got = orc.apply(psi0.copy(), dims, n, t, U)
        want = full_operator(U, dims, t) @ psi0
        assert np.abs(got - want).max() < 1e-13, op


@pytest.mark.parametrize("dc,dt", [(2, 4), (4, 2), (3, 5), (5, 3), (2, 3)])
def test_two_qudit_builders_block_structure(orc, dc, dt):
    X = orc.shift(dt, 1)
    want = sum(np.kron(np.diag(np.eye(dc)[c]), np.linalg.matrix_power(X, c)) for c in range(dc))
    assert np.abs(orc.sum_gate(dc, dt) - want).max() == 0
    assert np.abs(np.linalg.matrix_power(orc.sum_gate(dc, dt), dt) - np.eye(dc * dt)).max() < 1e-15
    th = 0.83
    for axis, j, k in [("x", 0, dt - 1), ("y", 0, 1), ("z", 0, 1), ("g", dt - 1, 0)]:
        want = sum(np.kron(np.diag(np.eye(dc)[m]), orc.rot(dt, j, k, m * th, axis)) for m in range(dc))
        assert np.abs(orc.crot(dc, j, k, th, axis, dt=dt) - want).max() < 1e-15
        h = 1e-6
        fd = (orc.crot(dc, j, k, th + h, axis, dt=dt) - orc.crot(dc, j, k, th - h, axis, dt=dt)) / (2 * h)
        assert np.abs(orc.crot_deriv(dc, j, k, th, axis, dt=dt) - fd).max() < 1e-8


@pytest.mark.parametrize("dims", DIMS)
def test_reductions_vs_numpy(orc, dims):
    n = len(dims)
    psi = rand_state(int(np.prod(dims)), 11)
    P = (np.abs(psi) ** 2).reshape(dims)
    e = orc.expect_number(psi, dims, n)
    for q in range(n):
        mq = P.sum(axis=tuple(a for a in range(n) if a != q))
        assert abs(e[q] - np.dot(np.arange(dims[q]), mq)) < 1e-13
    for idx in ([0], [n - 1, 0], [1, 2], list(range(n))[::-1]):
        got = orc.marginal(psi, dims, n, idx)
        rest = tuple(a for a in range(n) if a not in idx)
        m = P.sum(axis=rest) if rest else P
        kept = [a for a in range(n) if a in idx]
        m = np.transpose(m, [kept.index(a) for a in idx]).reshape(-1)
        assert np.abs(got - m).max() < 1e-14
    O = W.haar_unitary(dims[1], np.random.default_rng(3))
    O = O + O.conj().T
    got = orc.expect_obs(psi, dims, n, 1, O)
    want = np.vdot(psi, full_operator(O, dims, [1]) @ psi)
    assert abs(got - want) < 1e-13


@pytest.mark.parametrize("dims", DIMS + [[5, 2, 2, 3]])
def test_fourier_all_uniform(orc, dims):
    n = len(dims)
    psi = orc.run([W.Op("h", (q,)) for q in range(n)], dims, n)
    N = int(np.prod(dims))
    assert np.abs(psi - 1 / math.sqrt(N)).max() < 1e-15
    np.testing.assert_allclose(orc.expect_number(psi, dims, n), [(d - 1) / 2 for d in dims], atol=1e-14)


@pytest.mark.parametrize("dims", [[2, 3, 4], [3, 3, 5, 4], [2, 5]])
def test_ghz_ladder(orc, dims):
    """Fourier on the smallest qudit 0, then SUM(0, q): sum_m |m, m, ...>/sqrt(d_0)."""
    n = len(dims)
    ops = [W.Op("h", (0,))] + [W.Op("sum", (0, q)) for q in range(1, n)]
    psi = orc.run(ops, dims, n)
    d0 = dims[0]
    want = np.zeros(int(np.prod(dims)), dtype=np.complex128)
    for m in range(d0):
        want[np.ravel_multi_index([m] * n, dims)] = 1 / math.sqrt(d0)
    assert np.abs(psi - want).max() < 1e-15
    np.testing.assert_allclose(orc.expect_number(psi, dims, n), [(d0 - 1) / 2] * n, atol=1e-15)


def test_fourier_square_negates(orc):
    dims = [2, 3, 4, 5]
    n = len(dims)
    x = [1, 2, 3, 4]
    start = orc.basis(dims, n, int(np.ravel_multi_index(x, dims)))
    psi = orc.run([W.Op("h", (q,)) for q in range(n) for _ in range(2)], dims, n, psi=start)
    neg = [(-v) % d for v, d in zip(x, dims)]
    want = orc.basis(dims, n, int(np.ravel_multi_index(neg, dims)))
    assert np.abs(psi - want).max() < 1e-14
    psi4 = orc.run([W.Op("h", (q,)) for q in range(n) for _ in range(4)], dims, n, psi=start)
    assert np.abs(psi4 - start).max() < 1e-14


def test_code_style_example(orc):
    """dims [2, 3, 4] from |0, 1, 3>: Fourier on all, RX(pi/2) on qudit 0, CNOT(0, 2):
    every basis state ends with probability 1/24 and the marginal of qudits
    (0, 1) is uniform 1/6."""
    dims = [2, 3, 4]
    start = orc.basis(dims, 3, int(np.ravel_multi_index([0, 1, 3], dims)))
    ops = [W.Op("h", (0,)), W.Op("h", (1,)), W.Op("h", (2,)),
           W.Op("rot", (0,), j=0, k=1, axis="x", theta=math.pi / 2), W.Op("sum", (0, 2))]
    psi = orc.run(ops, dims, 3, psi=start)
    assert np.abs(np.abs(psi) ** 2 - 1 / 24).max() < 1e-15
    assert np.abs(orc.marginal(psi, dims, 3, [0, 1]) - 1 / 6).max() < 1e-15


def test_mixed_gradients_vs_fd(orc):
    dims = [2, 3, 4]
    ops, P = W.mixed_ansatz(dims, 2)
    theta = W.normal_angles(P, seed=41)
    w = [1.0, -0.5, 2.0]
    g = orc.grad_bruteforce(ops, dims, 3, theta, w)
    fd = orc.grad_fd(ops, dims, 3, theta, w)
    np.testing.assert_allclose(g, fd, atol=1e-8, rtol=1e-6)


def test_mixed_random_circuit_norm(orc):
    dims = [3, 2, 4, 3, 2]
    ops = W.mixed_random_circuit(dims, 120)
    assert {op.kind for op in ops} >= {"u", "rot", "z", "x", "h", "sum", "crot", "swap"}
    psi = orc.run(ops, dims, len(dims))
    assert abs(orc.norm2(psi) - 1) < 1e-13


def test_toffoli_qubits(orc):
    """d = 2, two controls: the textbook Toffoli truth table."""
    U = orc.mcx_gate([2, 2], 2)
    want = np.eye(8)
    want[[6, 7]] = want[[7, 6]]
    assert np.abs(U - want).max() == 0
    V = np.array([[0, 1], [1, 0]], dtype=complex)
    assert np.abs(orc.mcu_gate([2, 2], [1, 1], 2, V) - want).max() == 0


@pytest.mark.parametrize("dcs,dt", [([3], 3), ([2], 5), ([4], 3)])
def test_single_control_mcx_is_sum(orc, dcs, dt):
    assert np.abs(orc.mcx_gate(dcs, dt) - orc.sum_gate(dcs[0], dt)).max() == 0


@pytest.mark.parametrize("dcs,dt,s", [([3, 2], 4, 1), ([2, 3, 2], 3, 2), ([4, 4], 2, 1)])
def test_mcx_structure(orc, dcs, dt, s):
    """Block diagonal over control assignments with X_dt^(s * product) blocks;
    the dt-th power is the identity."""
    U = orc.mcx_gate(dcs, dt, s)
    X = orc.shift(dt, 1)
    want = np.zeros_like(U)
    for c, digs in enumerate(itertools.product(*[range(d) for d in dcs])):
        blk = np.linalg.matrix_power(X, (s * int(np.prod(digs))) % dt)
        want[c * dt:(c + 1) * dt, c * dt:(c + 1) * dt] = blk
    assert np.abs(U - want).max() == 0
    assert np.abs(np.linalg.matrix_power(U, dt) - np.eye(U.shape[0])).max() == 0


def test_mcu_structure(orc):
    dcs, levels, dt = [3, 2, 4], [2, 1, 0], 3
    V = W.haar_unitary(dt, np.random.default_rng(8))
    U = orc.mcu_gate(dcs, levels, dt, V)
    want = np.zeros_like(U)
    for c, digs in enumerate(itertools.product(*[range(d) for d in dcs])):
        want[c * dt:(c + 1) * dt, c * dt:(c + 1) * dt] = V if list(digs) == levels else np.eye(dt)
    assert np.abs(U - want).max() == 0


def test_mc_gates_on_register_vs_full_operator(orc):
    dims = [3, 2, 4, 3]
    psi0 = rand_state(int(np.prod(dims)), 9)
    V = W.haar_unitary(4, np.random.default_rng(2))
    for op in [W.Op("mcx", (0, 3, 2), power=1), W.Op("mcx", (2, 1, 0, 3), power=2),
               W.Op("mcu", (3, 0, 2), levels=(2, 1), matrix=V)]:
        t, U = orc.op_matrix(op, dims)
        got = orc.apply(psi0.copy(), dims, 4, t, U)
        assert np.abs(got - full_operator(U, dims, t) @ psi0).max() < 1e-14
