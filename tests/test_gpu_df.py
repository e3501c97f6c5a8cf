"""Complex128 programs in double-float arithmetic (the default for compiled
passes) against the oracle and against the same programs in FP64.

* Permutation gates only (shift X, SUM, SWAP): the gates are exact in both
  arithmetics, so the double-float result differs from the input's
  permutation only by the in-place conversion to hi + lo floats and back,
  at most 2^-48 relative per component; FP64 reproduces the oracle exactly.
* Random circuits of every gate kind the compiled passes handle, on random
  states: double-float and FP64 both within 1e-12 max-abs of the oracle.
* Amplitudes of very different magnitudes (1e-30 .. 1 and exact zeros):
  relative precision 2^-47 down to 2^-74, absolute 2^-96 below that (the low
  float would be subnormal), magnitudes below 2^-126 become 0.
* A program mixing compiled passes with a multi-controlled gate (an FP64
  kernel between double-float passes converts the state back and forth).
"""
import numpy as np
import pytest

from gpu_util import download, gpu_lib, upload
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(qf, ops, d, n, psi0, exact):
    st = upload(qf, psi0, d, n, "c128")
    p = qf.program_from_ops(d, n, ops)
    qf.qf_program_set_fp64(p, exact)
    qf.qf_program_run(p, st.handle)
    got = download(st)
    qf.qf_program_free(p)
    st.free()
    return got


@pytest.mark.parametrize("d,n", [(3, 9), (5, 6), (2, 14)])
def test_permutations_roundtrip(orc, d, n):
    qf = gpu_lib()
    rng = np.random.default_rng(d * 10 + n)
    ops = []
    for _ in range(60):
        k = rng.integers(3)
        if k == 0:
            ops.append(W.Op("x", (int(rng.integers(n)),), power=int(rng.integers(1, d))))
        else:
            c, t = (int(x) for x in rng.choice(n, 2, replace=False))
            ops.append(W.Op("sum" if k == 1 else "swap", (c, t)))
    psi0 = W.uniform_state(d, n, seed=n)
    want = orc.run(ops, d, n, psi0)
    exact = _run(qf, ops, d, n, psi0, True)
    assert np.array_equal(exact, want)
    df = _run(qf, ops, d, n, psi0, False)
    rel = max(np.abs(df.real - want.real).max() / np.abs(want.real).max(),
              np.abs(df.imag - want.imag).max() / np.abs(want.imag).max())
    err = np.abs(df - want) / np.maximum(np.abs(want), 1e-300)
    assert err.max() <= 2.0 ** -47, (err.max(), rel)


@pytest.mark.parametrize("d,n", [(2, 12), (3, 8), (4, 6), (5, 5), (7, 4)])
def test_random_circuits_both_arithmetics(orc, d, n):
    qf = gpu_lib()
    ops = W.random_circuit(d, n, 200, seed=d * 1000 + n)
    ops += [W.Op("rot", (0,), j=d - 1, axis="g", theta=0.4), W.Op("h", (n - 1,)),
            W.Op("crot", (n - 1, 0), j=0, k=1, axis="x", theta=1.1)]
    psi0 = W.uniform_state(d, n, seed=d + 2 * n)
    want = orc.run(ops, d, n, psi0)
    for exact in (False, True):
        got = _run(qf, ops, d, n, psi0, exact)
        err = np.abs(got - want).max()
        print("d=%d n=%d %s: max-abs %.3g" % (d, n, "fp64" if exact else "double-float", err))
        assert err <= 1e-12, (exact, err)


def test_magnitudes_and_zeros(orc):
    qf = gpu_lib()
    d, n = 3, 7
    rng = np.random.default_rng(3)
    N = d ** n
    mag = 10.0 ** rng.uniform(-30, 0, N)
    psi0 = mag * np.exp(2j * np.pi * rng.uniform(size=N))
    psi0[::17] = 0.0
    psi0[5] = 1e-40          # below 2^-126: becomes 0 in double-float form
    ops = [W.Op("x", (q,), power=1) for q in range(n)]   # exact permutation
    want = orc.run(ops, d, n, psi0)
    got = _run(qf, ops, d, n, psi0, False)
    moved = int(np.argmax(np.abs(want - 1e-40) < 1e-45))
    assert got[moved] == 0
    # each real component on its own: the double-float form splits components
    g = np.concatenate([got.real, got.imag])
    w = np.concatenate([want.real, want.imag])
    big = np.abs(w) >= 2.0 ** -74
    small = ~big & (np.abs(w) > 2.0 ** -126)
    assert np.all(g[w == 0] == 0)
    assert (np.abs(g[big] - w[big]) / np.abs(w[big])).max() <= 2.0 ** -47
    assert small.any() and np.abs(g[small] - w[small]).max() <= 2.0 ** -96


def test_multicontrolled_between_compiled_passes(orc):
    qf = gpu_lib()
    d, n = 3, 8
    ops = W.random_circuit(d, n, 60, seed=5)
    ops = ops[:30] + [W.Op("mcx", (0, 1, n - 1), power=1)] + ops[30:] + [W.Op("mcx", (2, 3, 4), power=2)]
    psi0 = W.uniform_state(d, n, seed=9)
    want = orc.run(ops, d, n, psi0)
    got = _run(qf, ops, d, n, psi0, False)
    assert np.abs(got - want).max() <= 1e-12


@pytest.mark.parametrize("d,n", [(3, 5), (2, 8), (5, 3), (4, 4)])
def test_adjoint_double_float_vs_fp64_and_oracle(orc, d, n):
    """The complex128 adjoint sweep with double-float reverse passes (default)
    and with FP64: gradients within 1e-10 of the oracle's derivative circuits,
    losses within 1e-12, psi restored to |0...0>."""
    qf = gpu_lib()
    ops, P = W.variational_ansatz(d, n, 3)
    ops = [W.Op("h", (q,)) for q in range(n)] + ops
    ops += [W.Op("crot", (0, n - 1), j=0, k=1, axis="y", param=0), W.Op("crot", (n - 1, 1), j=0, k=1, axis="z", param=1),
            W.Op("rot", (1,), j=d - 1, axis="g", param=2), W.Op("crot", (1, 0), j=1, axis="g", param=3),
            W.Op("swap", (0, 1))]
    theta = W.normal_angles(P, seed=d + n)
    w = np.linspace(0.5, 1.5, n)
    want = orc.grad_bruteforce(ops, d, n, theta, w)
    want_l = orc.loss(orc.run(ops, d, n, params=theta), d, n, w)
    for exact in (False, True):
        p = qf.program_from_ops(d, n, ops)
        qf.qf_program_set_fp64(p, exact)
        psi, lam = qf.State(d, n, "c128").set_basis(0), qf.State(d, n, "c128")
        loss, g = qf.qf_program_gradient(p, psi.handle, lam.handle, theta, w)
        back = download(psi)
        assert abs(loss - want_l) <= 1e-12, (exact, loss, want_l)
        assert np.abs(g - want).max() <= 1e-10, (exact, np.abs(g - want).max())
        e0 = np.zeros_like(back)
        e0[0] = 1.0
        assert np.abs(back - e0).max() <= 1e-12
        qf.qf_program_free(p)
        psi.free()
        lam.free()
