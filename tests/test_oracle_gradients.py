"""Pins of the oracle's gradient references (CPU only).

* One gate: RY^{01}(theta)|0> or RX^{01}(theta)|0> gives <N> = sin^2(theta/2), so
  dL/dtheta = sin(theta)/2 in closed form.
* Circuits of RZ gates only, started from a basis state, have zero gradient.
* Brute-force derivative circuits agree with central finite differences
  (h = 1e-5) on small ansatz circuits, including controlled rotations whose
  angle is scaled by the control level and parameters shared by several gates.
"""
import math

import numpy as np
import pytest

from paper_2409_17716_gb300 import workloads as W


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("d", [2, 3, 5])
def test_single_rotation_closed_form(orc, axis, d):
    ops = [W.Op("rot", (0,), j=0, k=1, axis=axis, param=0)]
    for th in (0.3, 1.7, 4.0):
        psi = orc.run(ops, d, 1, params=[th])
        assert abs(orc.expect_number(psi, d, 1)[0] - math.sin(th / 2) ** 2) < 1e-15
        g = orc.grad_bruteforce(ops, d, 1, [th], [1.0])
        assert abs(g[0] - math.sin(th) / 2) < 1e-14
        fd = orc.grad_fd(ops, d, 1, [th], [1.0])
        assert abs(fd[0] - math.sin(th) / 2) < 1e-9


def test_rz_only_zero_gradient(orc):
    d, n = 3, 3
    ops = [W.Op("rot", (q,), j=0, k=1, axis="z", param=q) for q in range(n)]
    ops += [W.Op("rot", (q,), j=1, k=2, axis="z", param=n + q) for q in range(n)]
    g = orc.grad_bruteforce(ops, d, n, np.linspace(0.1, 1.0, 2 * n), np.ones(n), psi0=orc.basis(d, n, 14))
    assert np.abs(g).max() < 1e-15


@pytest.mark.parametrize("d,n,layers", [(3, 3, 2), (2, 4, 2), (4, 2, 2)])
def test_bruteforce_vs_fd(orc, d, n, layers):
    ops, P = W.variational_ansatz(d, n, layers)
    ops = [W.Op("h", (q,)) for q in range(n)] + ops
    theta = W.normal_angles(P, seed=d * 10 + n)
    w = np.arange(1, n + 1, dtype=float)
    g = orc.grad_bruteforce(ops, d, n, theta, w)
    fd = orc.grad_fd(ops, d, n, theta, w, h=1e-5)
    np.testing.assert_allclose(g, fd, atol=1e-8, rtol=1e-6)


def test_shared_and_controlled_parameters(orc):
    """A parameter used by several gates (product rule) and controlled rotations."""
    d, n = 3, 3
    ops = [W.Op("h", (0,)), W.Op("h", (1,)),
           W.Op("crot", (0, 2), j=0, k=1, axis="y", param=0),
           W.Op("rot", (1,), j=1, k=2, axis="x", param=1),
           W.Op("crot", (1, 0), j=0, k=2, axis="x", param=0),
           W.Op("sum", (2, 1)),
           W.Op("rot", (2,), j=1, k=2, axis="g", param=1),
           W.Op("crot", (2, 1), j=1, k=2, axis="z", param=2)]
    theta = np.array([0.4, -1.1, 2.3])
    w = np.array([0.5, 1.0, -2.0])
    np.testing.assert_allclose(orc.grad_bruteforce(ops, d, n, theta, w),
                               orc.grad_fd(ops, d, n, theta, w), atol=1e-9)


@pytest.mark.parametrize("variant", ["R1", "R2", "R3"])
def test_vqa_variants_bruteforce_vs_fd(orc, variant):
    """The VQA circuit with each rotation block (RX, RY, level-pair RZ or
    Gell-Mann RZ, CNOT fan-out): derivative circuits agree with central
    differences."""
    d, n = 3, 3
    ops, P = W.vqa_circuit(d, n, variant, enc_first=0, theta_first=n)
    params = np.concatenate([np.linspace(0.2, 2.9, n), W.normal_angles(P, seed=P)])
    w = [1.0] + [0.0] * (n - 1)
    g = orc.grad_bruteforce(ops, d, n, params, w)
    fd = orc.grad_fd(ops, d, n, params, w)
    np.testing.assert_allclose(g, fd, atol=1e-8, rtol=1e-6)
