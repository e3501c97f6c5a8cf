"""Compiled tile passes (the default for programs) against the generic
interpreting tile kernel and the oracle: every gate kind in fused passes
(SWAP and custom two-qudit gates through shared memory, controls inside and
outside a register stage, multi-controlled passes in between), complex64 and
complex128, every d with a compiled stage layout (2-5) and one above it (7),
overridden stage slots, and a pass whose gate entries exceed the
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
