"""Compiled tile passes (the default for programs) against the generic
interpreting tile kernel and the oracle: every gate kind in fused passes
(SWAP and custom two-qudit gates through shared memory, controls inside and
outside a register stage, multi-controlled passes in between), complex64 and
complex128, every d with a compiled stage layout (2-5) and one above it (7),
overridden stage slots and tilings, and a pass whose gate entries exceed the
kernel-parameter budget (read from device memory instead)."""
import numpy as np
import pytest

from gpu_util import download, gpu_lib, tol
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def all_kinds(d, n, rng, gates=80):
    ops = W.random_circuit(d, n, gates, seed=d * 100 + n)
    extra = [W.Op("swap", (0, n - 1)), W.Op("u", (1, n - 2), matrix=W.haar_unitary(d * d, rng)) if d * d <= 64 else
             W.Op("sum", (1, n - 2)),
             W.Op("crot", (0, n - 1), j=0, k=d - 1, axis="x", theta=0.7),
             W.Op("crot", (n - 1, 0), j=0, k=1, axis="z", theta=-0.4),
             W.Op("crot", (n - 2, 1), j=d - 1, axis="g", theta=1.3),
             W.Op("rot", (2,), j=d - 1, axis="g", theta=0.3), W.Op("z", (3,), power=d - 1),
             W.Op("sum", (n - 1, 2)), W.Op("mcx", (0, 1, n - 1), power=1), W.Op("x", (1,), power=1)]
    return ops[:30] + extra + ops[30:]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("d,n", [(2, 12), (3, 8), (4, 6), (5, 5), (7, 4)])
def test_compiled_matches_generic_and_oracle(orc, d, n, dtype):
    qf = gpu_lib()
    ops = all_kinds(d, n, np.random.default_rng(d))
    want = orc.run(ops, d, n)
    p = qf.program_from_ops(d, n, ops)
    st = qf.State(d, n, dtype).set_basis(0)
    qf.qf_program_run(p, st.handle)
    jit = download(st)
    qf.qf_program_set_jit(p, False)
    st.set_basis(0)
    qf.qf_program_run(p, st.handle)
    gen = download(st)
    assert np.abs(jit - want).max() <= tol(dtype, len(ops))
    assert np.abs(gen - want).max() <= tol(dtype, len(ops))
    qf.qf_program_free(p)
    st.free()


@pytest.mark.parametrize("slots", [1, 2, 3, 4, 5])
def test_stage_slot_overrides(orc, slots):
    qf = gpu_lib()
    d, n = 2, 14
    ops = all_kinds(d, n, np.random.default_rng(2), gates=120)
    p = qf.program_from_ops(d, n, ops)
    qf.qf_program_set_stage_slots(p, slots)
    st = qf.State(d, n, "c64").set_basis(0)
    qf.qf_program_run(p, st.handle)
    assert np.abs(download(st) - orc.run(ops, d, n)).max() <= tol("c64", len(ops))
    qf.qf_program_free(p)
    st.free()


@pytest.mark.parametrize("d,n,dtype,tile,run", [
    (2, 16, "c64", 14, 0), (2, 16, "c64", 12, 4), (2, 15, "c128", 13, 0), (3, 11, "c64", 9, 0),
    (3, 10, "c128", 8, 2), (4, 9, "c64", 7, 1), (5, 8, "c64", 6, 2)])
def test_tiling_overrides(orc, d, n, dtype, tile, run):
    """Tile and run overrides up to the largest tile (160 KiB of amplitudes,
    where a second buffer no longer fits in a CTA's shared memory), compiled
    and generic."""
    qf = gpu_lib()
    ops = all_kinds(d, n, np.random.default_rng(d + 40))
    want = orc.run(ops, d, n)
    p = qf.program_from_ops(d, n, ops)
    qf.qf_program_set_tiling(p, tile, run, 0)
    st = qf.State(d, n, dtype)
    for jit in (True, False):
        qf.qf_program_set_jit(p, jit)
        st.set_basis(0)
        qf.qf_program_run(p, st.handle)
        assert np.abs(download(st) - want).max() <= tol(dtype, len(ops)), (jit, tile, run)
    qf.qf_program_free(p)
    st.free()


def test_entries_beyond_parameter_budget(orc):
    """96 controlled rotations of d=5 in one pass (20-25 entries each, not
    multiplied together): more entries than the kernel parameters hold, so
    the pass reads them from the program's buffer."""
    qf = gpu_lib()
    d, n = 5, 4
    rng = np.random.default_rng(9)
    ops = []
    for i in range(96):
        c, t = int(rng.integers(n)), int(rng.integers(n - 1))
        t = t + 1 if t >= c else t
        axis = "xyzg"[i % 4]
        j = 1 + i % (d - 1)
        ops.append(W.Op("crot", (c, t), j=0 if axis != "g" else j, k=j if axis != "g" else 1, axis=axis,
                        theta=float(rng.uniform(0, 6.28))))
    p = qf.program_from_ops(d, n, ops)
    src = qf.qf_program_jit_source(p)
    assert "A.gp[" in src
    for dtype in ("c64", "c128"):
        st = qf.State(d, n, dtype).set_basis(0)
        qf.qf_program_run(p, st.handle)
        assert np.abs(download(st) - orc.run(ops, d, n)).max() <= tol(dtype, len(ops))
        st.free()
    qf.qf_program_free(p)


def test_parameters_change_without_recompiling(orc):
    """Angles are passed per run: two parameter vectors through one compiled
    program both match the oracle."""
    qf = gpu_lib()
    d, n = 3, 7
    ops, P = W.variational_ansatz(d, n, 3)
    p = qf.program_from_ops(d, n, ops)
    st = qf.State(d, n, "c128")
    for seed in (1, 2):
        th = W.normal_angles(P, seed=seed)
        st.set_basis(0)
        qf.qf_program_run(p, st.handle, th)
        assert np.abs(download(st) - orc.run(ops, d, n, params=th)).max() <= 1e-12
    qf.qf_program_free(p)
    st.free()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("d,n", [(2, 10), (3, 7), (4, 5), (5, 4), (7, 3)])
def test_compiled_adjoint_matches_generic_and_oracle(orc, d, n, dtype):
    """Gradient of a circuit with every parametrised kind (level-pair and
    Gell-Mann rotations, controlled rotations with the control inside and
    outside a register stage, a parameter shared by several gates) between
    SWAP, custom two-qudit and multi-controlled gates: compiled reverse passes
    against the generic sweep and the oracle's derivative circuits."""
    qf = gpu_lib()
    rng = np.random.default_rng(d * 10 + n)
    ops = [W.Op("h", (q,)) for q in range(n)]
    slot = 0
    for q in range(n):
        ops.append(W.Op("rot", (q,), j=0, k=d - 1, axis="x", param=slot)); slot += 1
        ops.append(W.Op("rot", (q,), j=d - 1, axis="g", param=slot)); slot += 1
    ops += [W.Op("crot", (0, n - 1), j=0, k=1, axis="y", param=slot),
            W.Op("crot", (n - 1, 0), j=0, k=d - 1, axis="z", param=slot + 1),
            W.Op("swap", (0, n - 1)), W.Op("mcx", (0, 1, n - 1)),
            W.Op("crot", (1, n - 1), j=d - 1, axis="g", param=slot + 2),
            W.Op("rot", (n - 1,), j=0, k=1, axis="y", param=0)]
    if d * d <= 64:
        ops.append(W.Op("u", (1, 0), matrix=W.haar_unitary(d * d, rng)))
    ops.append(W.Op("crot", (n - 1, 1), j=0, k=1, axis="x", param=slot + 3))
    P = slot + 4
    theta = W.normal_angles(P, seed=P + d)
    w = np.linspace(0.5, 1.5, n)
    want = orc.grad_bruteforce(ops, d, n, theta, w)
    p = qf.program_from_ops(d, n, ops)
    psi, lam = qf.State(d, n, dtype), qf.State(d, n, dtype)
    grads = []
    for jit in (True, False):
        qf.qf_program_set_jit(p, jit)
        psi.set_basis(0)
        _, g = qf.qf_program_gradient(p, psi.handle, lam.handle, theta, w)
        grads.append(g)
    at = 1e-10 if dtype == "c128" else 1e-4 * max(1.0, np.abs(want).max())
    assert np.abs(grads[0] - want).max() <= at
    assert np.abs(grads[1] - want).max() <= at
    qf.qf_program_free(p)
    psi.free()
    lam.free()
