"""GPU parity of the batched forward and adjoint (qf_batch_*).

An uneven batch (d in 2..5, n in 4..10 or smaller, 2..6 layers; Fourier +
per-sample RZ encoding + shared-angle ansatz; loss <N_0>) is built once and run
through the captured graph.  Every circuit's loss and local gradient is
compared with the same circuit run alone through qf_program_gradient, a subset
of small circuits with the oracle (brute-force derivative circuits), and the
summed gradient with the sum of the per-circuit gradients.  A second run with
new parameters checks that the graph follows the parameter vector.
"""
import numpy as np
import pytest

from gpu_util import gpu_lib
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def make_batch(qf, circuits, params, dtype, weights_fn):
    b = qf.qf_batch_create(qf.QF_C64 if dtype == "c64" else qf.QF_C128)
    progs = []
    for c in circuits:
        p = qf.program_from_ops(c.d, c.n, c.ops)
        qf.qf_batch_add(b, p, weights_fn(c))
        progs.append(p)
    qf.qf_batch_build(b, len(params))
    return b, progs


def outputs(qf, b, ncirc, nlocal, nparams):
    loss, gl, gs = qf.qf_batch_read(b)
    assert len(loss) == ncirc
    return loss, gl, gs


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_matches_single_circuits(orc, dtype):
    qf = gpu_lib()
    circuits, params = W.batch_circuits(count=48, seed=123, n_range=(2, 7))
    w0 = lambda c: [1.0] + [0.0] * (c.n - 1)
    b, progs = make_batch(qf, circuits, params, dtype, w0)
    qf.qf_batch_run(b, params, True)
    info = qf.qf_batch_info(b)
    nlocal = sum(len(qf.qf_batch_circuit_params(b, i)[0]) for i in range(len(circuits)))
    loss, gl, gs = outputs(qf, b, len(circuits), nlocal, len(params))
    tol_l = 1e-12 if dtype == "c128" else 2e-6
    tol_g = 1e-10 if dtype == "c128" else 2e-5
    gsum = np.zeros(len(params))
    for i, c in enumerate(circuits):
        slots, off = qf.qf_batch_circuit_params(b, i)
        g_i = gl[off:off + len(slots)]
        gsum[slots] += g_i
        psi = qf.State(c.d, c.n, dtype)
        psi.set_basis(0)
        lam = qf.State(c.d, c.n, dtype)
        l1, g1 = qf.qf_program_gradient(progs[i], psi.handle, lam.handle, params, w0(c))
        psi.free()
        lam.free()
        assert abs(loss[i] - l1) <= tol_l, (i, loss[i], l1)
        assert np.abs(g_i - g1[slots]).max() <= tol_g, (i, np.abs(g_i - g1[slots]).max())
        if c.d ** c.n <= 800 and i % 3 == 0:
            want = orc.grad_bruteforce(c.ops, c.d, c.n, params, w0(c), slots=slots)
            assert np.abs(g_i - want).max() <= tol_g
            wl = orc.loss(orc.run(c.ops, c.d, c.n, params=params), c.d, c.n, w0(c))
            assert abs(loss[i] - wl) <= tol_l
    np.testing.assert_allclose(gs, gsum, atol=1e-12 * max(1, len(circuits)))
    # new parameters: the captured graph must follow them
    p2 = params + 0.37
    qf.qf_batch_run(b, p2, True)
    loss2, gl2, _ = outputs(qf, b, len(circuits), nlocal, len(params))
    for i in (0, len(circuits) // 2, len(circuits) - 1):
        c = circuits[i]
        slots, off = qf.qf_batch_circuit_params(b, i)
        psi = qf.State(c.d, c.n, dtype)
        psi.set_basis(0)
        lam = qf.State(c.d, c.n, dtype)
        l1, g1 = qf.qf_program_gradient(progs[i], psi.handle, lam.handle, p2, w0(c))
        psi.free()
        lam.free()
        assert abs(loss2[i] - l1) <= tol_l
        assert np.abs(gl2[off:off + len(slots)] - g1[slots]).max() <= tol_g
    # forward only
    qf.qf_batch_run(b, params, False)
    loss3, _, _ = outputs(qf, b, len(circuits), 0, 0)
    np.testing.assert_allclose(loss3, loss, atol=0)
    assert info["launches_backward"] > info["launches_forward"] > 0
    qf.qf_batch_free(b)
    for p in progs:
        qf.qf_program_free(p)


def _spread(slots, k=4):
    """k slots spread over a circuit's parameters (first, last, between)."""
    if len(slots) <= k:
        return list(slots)
    return [slots[int(round(i * (len(slots) - 1) / (k - 1)))] for i in range(k)]


def test_batch_full_size_sample(orc):
    """The 4096-circuit workload (d 2..5, n 4..10, L 2..6) in complex64: 16
    circuits drawn at random against the same circuit run alone (every
    parameter) and against the oracle (loss, and the derivative circuits of
    4 parameters per circuit: first, last and two between)."""
    qf = gpu_lib()
    circuits, params = W.batch_circuits(count=4096)
    w0 = lambda c: [1.0] + [0.0] * (c.n - 1)
    b, progs = make_batch(qf, circuits, params, "c64", w0)
    qf.qf_batch_run(b, params, True)
    nlocal = sum(len(qf.qf_batch_circuit_params(b, i)[0]) for i in range(len(circuits)))
    loss, gl, gs = outputs(qf, b, len(circuits), nlocal, len(params))
    rng = np.random.default_rng(0)
    for i in rng.choice(len(circuits), 16, replace=False):
        c = circuits[i]
        slots, off = qf.qf_batch_circuit_params(b, int(i))
        psi = qf.State(c.d, c.n, "c64")
        psi.set_basis(0)
        lam = qf.State(c.d, c.n, "c64")
        l1, g1 = qf.qf_program_gradient(progs[i], psi.handle, lam.handle, params, w0(c))
        psi.free()
        lam.free()
        assert abs(loss[i] - l1) <= 2e-6
        assert np.abs(gl[off:off + len(slots)] - g1[slots]).max() <= 2e-5
        sub = _spread(slots)
        want = orc.grad_bruteforce(c.ops, c.d, c.n, params, w0(c), slots=sub)
        got = np.array([gl[off + slots.index(s_)] for s_ in sub])
        assert np.abs(got - want).max() <= 2e-5, (int(i), np.abs(got - want).max())
        wl = orc.loss(orc.run(c.ops, c.d, c.n, params=params), c.d, c.n, w0(c))
        assert abs(loss[i] - wl) <= 2e-6
    assert np.isfinite(gs).all()
    qf.qf_batch_free(b)
    for p in progs:
        qf.qf_program_free(p)


def test_autotuned_batch_matches(tmp_path):
    """The autotuner picks a tile size and fusion depth per d from timed
    candidates; the tuned batch gives the same losses and gradients."""
    qf = gpu_lib()
    from paper_2409_17716_gb300 import autotune
    circuits, params = W.batch_circuits(count=24, seed=77, n_range=(3, 8))
    tuning = autotune.tune(circuits, params, qf.QF_C64, sample=4, cache_path=str(tmp_path / "tune.json"))
    assert set(tuning) == {c.d for c in circuits}
    for d, t in tuning.items():
        assert (t["tile_qudits"], t["max_ops"]) in autotune.candidates(d, False)
        assert len(t["tried"]) == len(autotune.candidates(d, False))
    w0 = lambda c: [1.0] + [0.0] * (c.n - 1)
    results = []
    for tuned in (False, True):
        b = qf.qf_batch_create(qf.QF_C64)
        progs = [qf.program_from_ops(c.d, c.n, c.ops) for c in circuits]
        for p, c in zip(progs, circuits):
            qf.qf_batch_add(b, p, w0(c))
        if tuned:
            autotune.apply(b, tuning)
        qf.qf_batch_build(b, len(params))
        qf.qf_batch_run(b, params, True)
        results.append(qf.qf_batch_read(b))
        qf.qf_batch_free(b)
        for p in progs:
            qf.qf_program_free(p)
    (l0, g0, s0), (l1, g1, s1) = results
    np.testing.assert_allclose(l1, l0, atol=2e-6)
    np.testing.assert_allclose(g1, g0, atol=2e-5)
    np.testing.assert_allclose(s1, s0, atol=1e-4)


@pytest.mark.parametrize("variant", ["R1", "R2", "R3"])
@pytest.mark.parametrize("d,n", [(3, 4), (10, 2)])
def test_vqa_batch_vs_oracle(orc, variant, d, n):
    """Batched VQA training step (Iris-like d=3 n=4, MNIST-like d=10 n=2):
    complex128 losses and per-sample gradients against the oracle."""
    qf = gpu_lib()
    circuits, params = W.vqa_batch(12, d, n, variant)
    w0 = lambda c: [1.0] + [0.0] * (c.n - 1)
    b, progs = make_batch(qf, circuits, params, "c128", w0)
    qf.qf_batch_run(b, params, True)
    loss, gl, gs = qf.qf_batch_read(b)
    for i in (0, 5, 11):
        c = circuits[i]
        slots, off = qf.qf_batch_circuit_params(b, i)
        want = orc.grad_bruteforce(c.ops, d, n, params, w0(c), slots=slots)
        assert np.abs(gl[off:off + len(slots)] - want).max() <= 1e-10
        wl = orc.loss(orc.run(c.ops, d, n, params=params), d, n, w0(c))
        assert abs(loss[i] - wl) <= 1e-12
    qf.qf_batch_free(b)
    for p in progs:
        qf.qf_program_free(p)


def test_batch_workload_prefix_c128_vs_oracle(orc):
    """The first 256 circuits of the 4096-circuit workload (same generator,
    n up to 10) batched in complex128: 16 of them, drawn at random, against
    the oracle -- loss within 1e-12, the derivative circuits of 4 parameters
    per circuit within 1e-10."""
    qf = gpu_lib()
    circuits, params = W.batch_circuits(count=4096)
    circuits = circuits[:256]
    assert max(c.n for c in circuits) == 10
    w0 = lambda c: [1.0] + [0.0] * (c.n - 1)
    b, progs = make_batch(qf, circuits, params, "c128", w0)
    qf.qf_batch_run(b, params, True)
    loss, gl, _ = qf.qf_batch_read(b)
    rng = np.random.default_rng(4)
    for i in rng.choice(len(circuits), 16, replace=False):
        c = circuits[i]
        slots, off = qf.qf_batch_circuit_params(b, int(i))
        sub = _spread(slots)
        want = orc.grad_bruteforce(c.ops, c.d, c.n, params, w0(c), slots=sub)
        got = np.array([gl[off + slots.index(s_)] for s_ in sub])
        assert np.abs(got - want).max() <= 1e-10, (int(i), np.abs(got - want).max())
        wl = orc.loss(orc.run(c.ops, c.d, c.n, params=params), c.d, c.n, w0(c))
        assert abs(loss[i] - wl) <= 1e-12, (int(i), loss[i], wl)
    qf.qf_batch_free(b)
    for p in progs:
        qf.qf_program_free(p)
