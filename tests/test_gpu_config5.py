"""Parity at the large-state size: d=3, n=20 (3.49e9 amplitudes, more than
2^31, so every 64-bit index path of the tile passes, the reductions and the
adjoint sweep is exercised at the size it was built for).

The host cannot hold the oracle's state at this size next to everything
else, so the checks are the ones the oracle and the mathematics fix at any
size:

* a 200-gate product circuit (gates of every benchmark kind inside three
  blocks of consecutive qudits): 4096 sampled amplitudes against the product
  of the oracle's block states, complex64 and complex128, and <N_q> of every
  qudit against the oracle's block expectations (a product state's marginal
  on a qudit is its block's marginal);
* the variational ansatz of the large-state adjoint workload (4 layers of
  RY, RZ on level pairs (0,1), (1,2) of every qudit and a SUM chain: 396
  gates, 320 parameters, loss sum_q <N_q>): the norm after the forward pass;
  the complex64 and complex128 losses against each other; the complex128
  adjoint gradient against FP64 central differences (h = 1e-5) of the
  complex128 forward (itself oracle-pinned at the benchmark sizes and by the
  product circuit above) on 32 parameters spread over all layers, relative
  error <= 1e-6; the complex64 adjoint gradient against the same
  differences (its error is stated, and bounded loosely).

The differences reuse prefixes: one complex128 state advances through the
circuit, and at each chosen parameter a copy runs the remaining gates at
theta +- h, so K parameters cost about K + 1 forward runs instead of 2K
(the complex128 forward runs in double-float arithmetic, about 1.7 s at this
size).
"""
import numpy as np
import pytest

from fullsize_util import bound, expected_product, product_circuit, sample_indices
from gpu_util import gpu_lib
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu

D, NQ, LAYERS = 3, 20, 4
# 32 parameters checked by finite differences: every layer, every rotation
# kind and qudits across the register (slot = layer*80 + kind*20 + qudit)
FD_SLOTS = sorted({(10 * i + 7 * (i % 4)) % 320 for i in range(32)} | {0, 319})[:32]


def _need(torch, gbytes):
    free, _ = torch.cuda.mem_get_info()
    assert free >= gbytes * 1e9, "needs %.0f GB of free device memory, %.0f GB free" % (gbytes, free / 1e9)


def _release(torch, *states):
    for st in states:
        st.free()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_product_circuit_n20_sampled(orc, dtype):
    import torch
    qf = gpu_lib()
    d, n, gates = D, NQ, 200
    _need(torch, (8 if dtype == "c64" else 16) * d ** n / 1e9 + 4)
    full, local, blocks = product_circuit(d, n, gates, seed=20)
    states = [orc.run(ops, d, hi - lo) for ops, (lo, hi) in zip(local, blocks)]
    p = qf.program_from_ops(d, n, full, fuse=True)
    st = qf.State(d, n, dtype).set_basis(0)
    qf.qf_program_run(p, st.handle)
    torch.cuda.synchronize()
    idx = sample_indices(d, n, 4096, seed=20)
    assert idx.max() >= 2 ** 31
    got = st.tensor[torch.from_numpy(idx).to("cuda")].cpu().numpy().astype(np.complex128)
    want = expected_product(states, blocks, d, n, idx)
    e = st.expect_number()
    want_e = np.concatenate([orc.expect_number(s, d, hi - lo) for s, (lo, hi) in zip(states, blocks)])
    if dtype == "c64":
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert rel <= bound(d, gates), rel
        assert abs(e[n] - 1.0) <= 2 * bound(d, gates)
        assert np.abs(e[:n] - want_e).max() <= 2 * bound(d, gates) * (d - 1)
    else:
        assert np.abs(got - want).max() <= 1e-12
        assert abs(e[n] - 1.0) <= 1e-12
        assert np.abs(e[:n] - want_e).max() <= 1e-11
    qf.qf_program_free(p)
    _release(torch, st)


def _loss(qf, st, w):
    return float(np.dot(w, st.expect_number()[:len(w)]))


def test_ansatz_n20_adjoint_vs_finite_differences():
    import torch
    qf = gpu_lib()
    d, n = D, NQ
    N = d ** n
    ops, P = W.variational_ansatz(d, n, LAYERS, entangler="chain")
    assert P == 320 and len(ops) == 396
    theta = W.normal_angles(P, seed=n)
    w = np.ones(n)
    pos = {op.param: l for l, op in enumerate(ops) if op.param >= 0}

    # complex64: forward norm, then loss and full gradient (psi, lambda)
    _need(torch, 2 * 8 * N / 1e9 + 4)
    p = qf.program_from_ops(d, n, ops)
    psi, lam = qf.State(d, n, "c64").set_basis(0), qf.State(d, n, "c64")
    qf.qf_program_run(p, psi.handle, theta)
    e = psi.expect_number()
    assert abs(e[n] - 1.0) <= 2 * bound(d, len(ops))
    loss_fwd64 = float(np.dot(w, e[:n]))
    psi.set_basis(0)
    loss64, g64 = qf.qf_program_gradient(p, psi.handle, lam.handle, theta, w)
    assert abs(loss64 - loss_fwd64) <= 1e-9 * abs(loss_fwd64)
    # the sweep uncomputes psi back to |0...0>
    back0 = complex(psi.tensor[0].item())
    assert abs(back0 - 1.0) <= 4 * bound(d, len(ops))
    _release(torch, psi, lam)

    # complex128: loss and full gradient
    _need(torch, 2 * 16 * N / 1e9 + 4)
    a, b = qf.State(d, n, "c128").set_basis(0), qf.State(d, n, "c128")
    loss128, g128 = qf.qf_program_gradient(p, a.handle, b.handle, theta, w)
    qf.qf_program_free(p)
    print("n=20 loss: complex64 %.12f complex128 %.12f" % (loss64, loss128))
    assert abs(loss64 - loss128) <= 1e-5 * abs(loss128)

    # FP64 central differences of the complex128 forward on FD_SLOTS, with
    # one cursor state (a) and a working copy (b)
    h = 1e-5
    slots = sorted(FD_SLOTS, key=lambda s: pos[s])
    a.set_basis(0)
    prev = 0
    fd = {}
    for s in slots:
        l = pos[s]
        if l > prev:
            seg = qf.program_from_ops(d, n, ops[prev:l])
            qf.qf_program_run(seg, a.handle, theta)
            qf.qf_program_free(seg)
            prev = l
        suf = qf.program_from_ops(d, n, ops[l:])
        vals = []
        for sign in (1.0, -1.0):
            b.tensor.copy_(a.tensor)
            t = theta.copy()
            t[s] += sign * h
            qf.qf_program_run(suf, b.handle, t)
            vals.append(_loss(qf, b, w))
        qf.qf_program_free(suf)
        fd[s] = (vals[0] - vals[1]) / (2 * h)
    _release(torch, a, b)

    err128 = max(abs(g128[s] - fd[s]) / max(1.0, abs(fd[s])) for s in slots)
    err64 = max(abs(g64[s] - fd[s]) / max(1.0, abs(fd[s])) for s in slots)
    print("n=20 adjoint vs central differences (relative to max(1,|fd|)): complex128 %.3g complex64 %.3g"
          % (err128, err64))
    print("n=20 complex64 vs complex128 adjoint, all %d parameters: max-abs %.3g" % (P, np.abs(g64 - g128).max()))
    for s in slots:
        assert abs(g128[s] - fd[s]) <= 1e-6 * max(1.0, abs(fd[s])), (s, g128[s], fd[s])
        assert abs(g64[s] - fd[s]) <= 1e-4 * max(1.0, abs(fd[s])), (s, g64[s], fd[s])
    assert np.abs(g64 - g128).max() <= 1e-4 * max(1.0, np.abs(g128).max())
