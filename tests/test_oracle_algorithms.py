"""Closed-form pins of whole oracle circuits (CPU only).

* Fourier on every qudit of |0..0> gives amplitudes d^(-n/2) and <N_q> = (d-1)/2.
* Fourier on qudit 0 then the SUM chain gives the GHZ state sum_m |m..m>/sqrt(d).
* SUM^d = I on registers, norm preservation over random circuits, a level-pair
  RZ on a basis state is a pure phase.
* Deutsch-Jozsa for qudits (Results, Deutsch-Jozsa algorithm): with input
  |0, 0, 0, d-1>, the constant oracle (X on the last qudit) leaves the register
  at |000> with probability 1; the balanced oracle CNOT(2, 3) kicks the phase
  w^c back onto register qudit 2, which ends in |d-1> with probability 1.
* Grover for two qutrits (Results, Grover's algorithm): one oracle + diffusion
  iteration over 9 items marks |22> with probability sin^2(3 arcsin(1/3)).
"""
import math

import numpy as np
import pytest

from paper_2409_17716_gb300 import workloads as W


@pytest.mark.parametrize("d,n", [(2, 6), (3, 5), (4, 4), (5, 3), (7, 2)])
def test_uniform_superposition(orc, d, n):
    ops = [W.Op("h", (q,)) for q in range(n)]
    psi = orc.run(ops, d, n)
    np.testing.assert_allclose(psi, np.full(d ** n, d ** (-n / 2)), atol=1e-14)
    np.testing.assert_allclose(orc.expect_number(psi, d, n), np.full(n, (d - 1) / 2), atol=1e-13)


@pytest.mark.parametrize("d,n", [(2, 6), (3, 5), (4, 4), (5, 3)])
def test_ghz(orc, d, n):
    ops = [W.Op("h", (0,))] + [W.Op("sum", (q, q + 1)) for q in range(n - 1)]
    psi = orc.run(ops, d, n)
    want = np.zeros(d ** n, dtype=complex)
    rep = (d ** n - 1) // (d - 1)
    for m in range(d):
        want[m * rep] = 1 / math.sqrt(d)
    np.testing.assert_allclose(psi, want, atol=1e-14)
    np.testing.assert_allclose(orc.expect_number(psi, d, n), np.full(n, (d - 1) / 2), atol=1e-13)


def test_sum_power_identity_and_norm(orc):
    d, n = 3, 4
    psi0 = W.uniform_state(d, n, seed=9)
    ops = [W.Op("sum", (2, 0))] * d
    np.testing.assert_allclose(orc.run(ops, d, n, psi0), psi0, atol=1e-15)
    circ = W.random_circuit(d, n, 60, seed=99)
    psi = orc.run(circ, d, n, psi0)
    assert abs(orc.norm2(psi) - 1) < 1e-13


def test_rz_on_basis_is_phase(orc):
    d, n = 4, 3
    for idx in (0, 5, 37):
        psi0 = orc.basis(d, n, idx)
        ops = [W.Op("rot", (q,), j=j, k=k, axis="z", theta=0.3 + q) for q in range(n) for (j, k) in [(0, 1), (1, 3)]]
        ops += [W.Op("rot", (1,), j=2, axis="g", theta=1.2), W.Op("z", (2,), power=3)]
        psi = orc.run(ops, d, n, psi0)
        assert abs(abs(psi[idx]) - 1) < 1e-14
        np.testing.assert_allclose(orc.expect_number(psi, d, n), orc.expect_number(psi0, d, n), atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
@pytest.mark.parametrize("mode", ["constant", "balanced"])
def test_deutsch_jozsa(orc, d, mode):
    n = 4
    start = (d - 1)  # |0, 0, 0, d-1>
    ops = [W.Op("h", (q,)) for q in range(n)]
    ops.append(W.Op("x", (n - 1,)) if mode == "constant" else W.Op("sum", (2, 3)))
    ops += [W.Op("h", (q,)) for q in range(n - 1)]
    psi = orc.run(ops, d, n, orc.basis(d, n, start))
    reg = orc.marginal(psi, d, n, [0, 1, 2])
    expect = 0 if mode == "constant" else d - 1  # register index (0, 0, x)
    assert abs(reg[expect] - 1) < 1e-12


def test_grover_two_qutrits(orc):
    d, n = 3, 2
    N = d ** n
    s = orc.run([W.Op("h", (0,)), W.Op("h", (1,))], d, n)
    marked = np.zeros(N, dtype=complex)
    marked[2 * d + 2] = 1
    oracle_u = np.eye(N) - 2 * np.outer(marked, marked.conj())
    diffusion = 2 * np.outer(s, s.conj()) - np.eye(N)
    ops = [W.Op("u", (0, 1), matrix=oracle_u), W.Op("u", (0, 1), matrix=diffusion)]
    out = orc.run(ops, d, n, s)
    p = np.abs(out) ** 2
    want = math.sin(3 * math.asin(1 / 3)) ** 2
    assert abs(p[8] - want) < 1e-14
    assert abs(want - 0.7256515775034293) < 1e-15
