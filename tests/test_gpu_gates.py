"""GPU parity of every gate kind at every target position, through the C ABI.

For each (d, n, dtype) a random state is uploaded, one kind of gate is applied
at every target (and every ordered control/target pair), and the result is
compared element by element with the oracle applying the same gates to the
same state.  Sizes cover strides below and above one warp (tile and strided
kernels), several tiles per state, templated d = 2..8 and the generic path
(d = 9, 16), and n = 1.
"""
import itertools

import numpy as np
import pytest

from gpu_util import download, gpu_lib, tol, upload
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [(2, 10), (2, 15), (3, 7), (3, 10), (4, 5), (4, 8), (5, 4), (5, 6), (6, 4), (7, 3), (8, 3), (9, 3), (16, 2),
         (3, 1), (2, 1)]


def kind_ops(kind, d, n, rng):
    ops = []
    pairs = [(j, k) for j in range(d) for k in range(j + 1, d)]
    if kind == "h":
        ops = [W.Op("h", (q,)) for q in range(n)]
    elif kind == "x":
        ops = [W.Op("x", (q,), power=p) for q in range(n) for p in (1, d - 1, 2 * d + 1)]
    elif kind == "z":
        ops = [W.Op("z", (q,), power=p) for q in range(n) for p in (1, d - 1, 3)]
    elif kind in ("rx", "ry", "rz"):
        ops = [W.Op("rot", (q,), j=j, k=k, axis=kind[1], theta=float(rng.uniform(0, 2 * np.pi)))
               for q in range(n) for (j, k) in pairs[:4] + pairs[-1:]]
    elif kind == "rg":
        ops = [W.Op("rot", (q,), j=j, axis="g", theta=float(rng.uniform(0, 2 * np.pi)))
               for q in range(n) for j in range(1, d)]
    elif kind == "u":
        ops = [W.Op("u", (q,), matrix=W.haar_unitary(d, rng)) for q in range(n)]
    elif kind == "sum":
        ops = [W.Op("sum", (c, t)) for c, t in itertools.permutations(range(n), 2)]
    elif kind == "swap":
        ops = [W.Op("swap", (c, t)) for c, t in itertools.permutations(range(n), 2)]
    elif kind.startswith("cr"):
        ax = kind[2]
        ops = []
        for c, t in itertools.permutations(range(n), 2):
            if ax == "g":
                ops.append(W.Op("crot", (c, t), j=int(rng.integers(1, d)), axis="g", theta=float(rng.uniform(0, 6))))
            else:
                j, k = pairs[int(rng.integers(len(pairs)))]
                ops.append(W.Op("crot", (c, t), j=j, k=k, axis=ax, theta=float(rng.uniform(0, 6))))
    elif kind == "u2":
        if d ** 2 > 64:
            return []
        ops = [W.Op("u", (c, t), matrix=W.haar_unitary(d * d, rng)) for c, t in itertools.permutations(range(n), 2)][:12]
    return ops


CHUNK = 200
KINDS = ["h", "x", "z", "rx", "ry", "rz", "rg", "u", "sum", "swap", "crx", "cry", "crz", "crg", "u2"]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("d,n", SIZES)
def test_every_kind_every_target(orc, d, n, dtype):
    qf = gpu_lib()
    rng = np.random.default_rng(1000 * d + n)
    psi0 = W.uniform_state(d, n, seed=d + n)
    for kind in KINDS:
        ops = kind_ops(kind, d, n, rng)
        if n < 2 and kind in ("sum", "swap", "crx", "cry", "crz", "crg", "u2"):
            continue
        if not ops:
            continue
        # at most 200 gates per comparison (the stated tolerances are per
        # 200-gate circuit); each chunk starts from the oracle's state
        psi_in = psi0
        for c0 in range(0, len(ops), CHUNK):
            chunk = ops[c0:c0 + CHUNK]
            st = upload(qf, psi_in, d, n, dtype)
            qf.apply_ops(st.handle, chunk)
            got = download(st)
            want = orc.run(chunk, d, n, psi_in)
            err = np.abs(got - want).max()
            assert err <= tol(dtype, len(chunk)), "%s d=%d n=%d %s gates %d..: err %.3g" % (kind, d, n, dtype, c0, err)
            st.free()
            psi_in = want


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_canary_untouched(orc, dtype):
    """A state wrapped inside a larger buffer: the guard regions before and
    after it stay bit-identical through every kind of gate."""
    import torch
    qf = gpu_lib()
    d, n = 3, 9   # odd N
    N = d ** n
    pad = 64
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    buf = torch.full((N + 2 * pad,), complex(7.0, -3.0), dtype=tdt, device="cuda")
    psi0 = W.uniform_state(d, n, seed=3)
    buf[pad:pad + N] = torch.from_numpy(psi0).to(buf)
    st = qf.State(d, n, dtype, tensor=buf[pad:pad + N])
    rng = np.random.default_rng(5)
    ops = []
    for kind in KINDS:
        ops += kind_ops(kind, d, n, rng)[:6]
    qf.apply_ops(st.handle, ops)
    p = qf.program_from_ops(d, n, ops, fuse=True)
    qf.qf_program_run(p, st.handle)
    qf.qf_program_free(p)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert np.all(b[:pad] == complex(7.0, -3.0)) and np.all(b[pad + N:] == complex(7.0, -3.0))
    want = orc.run(ops + ops, d, n, psi0)
    assert np.abs(b[pad:pad + N] - want).max() <= tol(dtype, 200)
    st.free()


def test_invalid_gate_leaves_state(orc):
    qf = gpu_lib()
    d, n = 3, 5
    psi0 = W.uniform_state(d, n, seed=8)
    st = upload(qf, psi0, d, n, "c128")
    bad = [lambda: qf.qf_apply_rot(st.handle, 5, 0, 1, 0.3, "x"),
           lambda: qf.qf_apply_rot(st.handle, 0, 2, 1, 0.3, "y"),
           lambda: qf.qf_apply_crot(st.handle, 1, 1, 0, 1, 0.3, "y"),
           lambda: qf.qf_apply_sum(st.handle, 0, 5),
           lambda: qf.qf_apply_gate(st.handle, [0, 0], np.eye(9))]
    for f in bad:
        with pytest.raises(qf.QFError) as ei:
            f()
        assert ei.value.status == qf.QF_ERR_ARG
    assert np.array_equal(download(st), psi0)
    st.free()


def test_owned_state_init_and_basis(orc):
    qf = gpu_lib()
    import ctypes
    import torch
    for d, n, dt in [(3, 5, qf.QF_C64), (2, 7, qf.QF_C128)]:
        h = qf.qf_state_init(d, n, dt)
        ptr, N = qf.qf_state_ptr(h)
        assert N == d ** n
        assert qf.qf_state_info(h) == (d, n, dt)
        e = qf.qf_expect(h, qf.QF_OBS_NUMBER_ALL)
        np.testing.assert_allclose(e, [0.0] * n + [1.0], atol=0)
        idx = N - 2
        qf.qf_state_set_basis(h, idx)
        e = qf.qf_expect(h, qf.QF_OBS_NUMBER_ALL)
        want = orc.expect_number(orc.basis(d, n, idx), d, n)
        np.testing.assert_allclose(e[:n], want, atol=0)
        qf.qf_state_free(h)
