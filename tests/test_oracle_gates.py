"""Pins of the oracle's gate builders (CPU only).

Each builder is checked against something other than itself:
* the matrices the paper prints (tests/golden/paper_gate_matrices.json),
* matrix exponentials exp(-i theta S / 2) of generators written out here from
  the paper's Gell-Mann definitions (scipy.linalg.expm),
* textbook qubit gates at d = 2 (Hadamard, Pauli X/Z, CNOT, RX/RY/RZ, CRY),
* algebraic invariants (unitarity, X^d = I, Z^d = I, ZX = wXZ, H X H^+ = Z,
  H^4 = I, H^2|x> = |-x>, SUM^d = I, Gell-Mann orthonormality).
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_gate_matrices.json")
THETAS = [0.0, 0.37, 1.3, math.pi, 2.9, 5.1, -0.8]


def _eval(sym, D, theta):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    w = cmath.exp(2j * math.pi / D)
    env = {"c": c, "s": s, "r": 1 / math.sqrt(D), "w": w, "i": 1j,
           "e-": cmath.exp(-0.5j * theta), "e+": cmath.exp(0.5j * theta)}
    if sym in env:
        return env[sym]
    if sym == "-is":
        return -1j * s
    if sym == "-s":
        return -s
    if sym == "-i":
        return -1j
    if sym == "-1":
        return -1.0
    if sym.startswith("r*w^"):
        return env["r"] * w ** int(sym[4:])
    if sym == "r*w":
        return env["r"] * w
    if sym.startswith("w^"):
        return w ** int(sym[2:])
    return complex(float(sym))


def _gold_cases():
    with open(GOLD) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _gold_cases()["cases"], ids=lambda c: c["cite"])
def test_printed_matrices(orc, case):
    D = case["D"]
    for th in THETAS:
        want = np.array([[_eval(x, D, th) for x in row] for row in case["matrix"]])
        g = case["gate"]
        if g == "rot":
            got = orc.rot(D, case["j"], case["k"], th, case["axis"])
        elif g == "gen":
            got = orc.generator(D, case["j"], case["k"], case["axis"])
        elif g == "fourier":
            got = orc.fourier(D)
        elif g == "phase":
            got = orc.clock(D, 1)
        else:
            raise AssertionError(g)
        np.testing.assert_allclose(got, want, atol=1e-14, rtol=0, err_msg=case["cite"])


def test_printed_not_transitions(orc):
    t = _gold_cases()["transitions"]
    X = orc.shift(t["D"], t["s"])
    for a, b in t["map"]:
        e = np.zeros(t["D"]); e[a] = 1
        out = X @ e
        assert np.argmax(np.abs(out)) == b and abs(out[b] - 1) < 1e-15


def _gellmann(d, j, k, axis):
    """Generators written out from the paper's definitions (0-based levels)."""
    S = np.zeros((d, d), dtype=complex)
    ket = lambda a: np.eye(d)[:, [a]]
    if axis == "x":
        S = ket(j) @ ket(k).T + ket(k) @ ket(j).T
    elif axis == "y":
        S = -1j * ket(j) @ ket(k).T + 1j * ket(k) @ ket(j).T
    elif axis == "z":
        S = ket(j) @ ket(j).T - ket(k) @ ket(k).T
    elif axis == "g":
        S = sum(ket(l) @ ket(l).T for l in range(j)) - j * ket(j) @ ket(j).T
        S = math.sqrt(2.0 / (j * (j + 1))) * S
    return S.astype(complex)


def _all_rotations(d):
    for j in range(d):
        for k in range(j + 1, d):
            for axis in "xyz":
                yield j, k, axis
    for j in range(1, d):
        yield j, 0, "g"


@pytest.mark.parametrize("d", [2, 3, 4, 5, 7])
def test_rotation_is_matrix_exponential(orc, d):
    from scipy.linalg import expm
    for j, k, axis in _all_rotations(d):
        S = _gellmann(d, j, k, axis)
        np.testing.assert_allclose(orc.generator(d, j, k, axis), S, atol=1e-15)
        for th in THETAS:
            want = expm(-0.5j * th * S)
            np.testing.assert_allclose(orc.rot(d, j, k, th, axis), want, atol=1e-13)
            # derivative of exp(-i theta S/2) by central differences of expm
            h = 1e-6
            fd = (expm(-0.5j * (th + h) * S) - expm(-0.5j * (th - h) * S)) / (2 * h)
            np.testing.assert_allclose(orc.rot_deriv(d, j, k, th, axis), fd, atol=1e-8)


@pytest.mark.parametrize("d", [2, 3, 4, 6])
def test_gellmann_orthonormal(orc, d):
    """Generalised Gell-Mann matrices: Hermitian, traceless, Tr(S_a S_b) = 2 delta_ab."""
    gens = [orc.generator(d, j, k, a) for (j, k, a) in _all_rotations(d) if a != "z"]
    assert len(gens) == d * d - 1
    for A in gens:
        np.testing.assert_allclose(A, A.conj().T, atol=1e-15)
        assert abs(np.trace(A)) < 1e-14
    G = np.array([[np.trace(A @ B) for B in gens] for A in gens])
    np.testing.assert_allclose(G, 2 * np.eye(len(gens)), atol=1e-13)


def test_qubit_reductions(orc):
    """d = 2 gives the textbook qubit gates."""
    s2 = 1 / math.sqrt(2)
    np.testing.assert_allclose(orc.fourier(2), [[s2, s2], [s2, -s2]], atol=1e-15)
    np.testing.assert_allclose(orc.shift(2), [[0, 1], [1, 0]], atol=0)
    np.testing.assert_allclose(orc.clock(2), [[1, 0], [0, -1]], atol=1e-15)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])
    np.testing.assert_allclose(orc.sum_gate(2), cnot, atol=0)
    for th in THETAS:
        c, s = math.cos(th / 2), math.sin(th / 2)
        rx = np.array([[c, -1j * s], [-1j * s, c]])
        ry = np.array([[c, -s], [s, c]])
        rz = np.diag([cmath.exp(-0.5j * th), cmath.exp(0.5j * th)])
        np.testing.assert_allclose(orc.rot(2, 0, 1, th, "x"), rx, atol=1e-15)
        np.testing.assert_allclose(orc.rot(2, 0, 1, th, "y"), ry, atol=1e-15)
        np.testing.assert_allclose(orc.rot(2, 0, 1, th, "z"), rz, atol=1e-15)
        cry = np.eye(4, dtype=complex)
        cry[2:, 2:] = ry
        np.testing.assert_allclose(orc.crot(2, 0, 1, th, "y"), cry, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 8])
def test_invariants(orc, d):
    I = np.eye(d)
    w = cmath.exp(2j * math.pi / d)
    X, Z, H = orc.shift(d, 1), orc.clock(d, 1), orc.fourier(d)
    for U in [X, Z, H, orc.shift(d, d - 1), orc.clock(d, 2)]:
        np.testing.assert_allclose(U.conj().T @ U, I, atol=1e-13)
    np.testing.assert_allclose(np.linalg.matrix_power(X, d), I, atol=1e-13)
    np.testing.assert_allclose(np.linalg.matrix_power(Z, d), I, atol=1e-12)
    np.testing.assert_allclose(Z @ X, w * X @ Z, atol=1e-13)
    np.testing.assert_allclose(H @ X @ H.conj().T, Z, atol=1e-13)
    np.testing.assert_allclose(np.linalg.matrix_power(H, 4), I, atol=1e-12)
    H2 = H @ H
    for x in range(d):
        e = I[:, x]
        np.testing.assert_allclose(H2 @ e, I[:, (-x) % d], atol=1e-13)
    # H|0> is the equal superposition of all d levels
    np.testing.assert_allclose(H[:, 0], np.full(d, 1 / math.sqrt(d)), atol=1e-15)
    for s in range(d + 2):
        np.testing.assert_allclose(orc.shift(d, s), np.linalg.matrix_power(X, s), atol=1e-13)
    S = orc.sum_gate(d)
    np.testing.assert_allclose(np.linalg.matrix_power(S, d), np.eye(d * d), atol=0)
    W = orc.swap_gate(d)
    np.testing.assert_allclose(W @ W, np.eye(d * d), atol=0)
    for j, k, axis in _all_rotations(d):
        for th in THETAS:
            R = orc.rot(d, j, k, th, axis)
            np.testing.assert_allclose(R.conj().T @ R, I, atol=1e-13)
            if axis in "xyz":  # two-level generators have eigenvalues +-1, 0
                np.testing.assert_allclose(orc.rot(d, j, k, th + 4 * math.pi, axis), R, atol=1e-12)
        if axis in "xyz":
            R = orc.rot(d, j, k, 2 * math.pi, axis)
            want = np.eye(d, dtype=complex)
            want[j, j] = want[k, k] = -1
            np.testing.assert_allclose(R, want, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_controlled_rotation_blocks(orc, d):
    """sum_m |m><m| (x) R(m theta): control level m carries R(m theta); m = 0 is identity."""
    for j, k, axis in _all_rotations(d):
        for th in (0.3, 2.2):
            C = orc.crot(d, j, k, th, axis)
            np.testing.assert_allclose(C.conj().T @ C, np.eye(d * d), atol=1e-13)
            for m in range(d):
                for m2 in range(d):
                    blk = C[m * d:(m + 1) * d, m2 * d:(m2 + 1) * d]
                    if m == m2:
                        np.testing.assert_allclose(blk, orc.rot(d, j, k, m * th, axis), atol=1e-14)
                    else:
                        assert np.abs(blk).max() == 0
            h = 1e-6
            fd = (orc.crot(d, j, k, th + h, axis) - orc.crot(d, j, k, th - h, axis)) / (2 * h)
            np.testing.assert_allclose(orc.crot_deriv(d, j, k, th, axis), fd, atol=1e-8)


def test_sum_index_rule(orc):
    """<c, t (+) c| SUM |c, t> = 1 and all other entries 0 (Generalized CNOT gate)."""
    for d in (2, 3, 5):
        S = orc.sum_gate(d)
        for c in range(d):
            for t in range(d):
                col = c * d + t
                assert S[c * d + (t + c) % d, col] == 1
                assert np.count_nonzero(S[:, col]) == 1


def test_invalid_arguments(orc):
    with pytest.raises(ValueError):
        orc.rot(3, 1, 1, 0.1, "x")
    with pytest.raises(ValueError):
        orc.rot(3, 0, 3, 0.1, "y")
    with pytest.raises(ValueError):
        orc.rot(3, 0, 1, 0.1, "q")
    with pytest.raises(ValueError):
        orc.rot(3, 3, 0, 0.1, "g")
