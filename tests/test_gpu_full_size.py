"""Parity at the benchmark's full sizes (d=2 n=28, d=3 n=17, d=4 n=14,
d=5 n=12, complex64), in the launch configuration the benchmark times: fused
programs with compiled tile passes and default tiling, run through the C ABI.

A full state is too large for the oracle, so two checks that it can make at
any size:

* Product circuits.  Random gates of every kind the benchmark draws, each
  confined to one of three blocks of consecutive qudits, so the final state
  is the tensor product of three block states.  The oracle computes each
  block state; every sampled amplitude of the full state must equal the
  product of the three block amplitudes at the index's block digits (basis
  index i = sum_q i_q d^(n-1-q), qudit 0 most significant).
* The benchmark's own 200-gate sequences followed by their inverse (each
  gate's inverse, in reverse order) must return |0...0>, and the norm must
  be 1 after the forward half.

Tolerance: a complex64 d-term dot product per gate and amplitude adds at
most about 2 d 2^-24 relative error, so after G gates the error vector's
norm is below 2 G d 2^-24; the tests allow twice that, for the round trip's
distance from |0...0> and, relative to the sampled amplitudes' norm, for the
sampled amplitudes (rounding spreads over the amplitudes like the state
does, while a wrong gate, index or level gives relative errors of order 1).
"""
import numpy as np
import pytest

from gpu_util import gpu_lib
from paper_2409_17716_gb300 import workloads as W

SIZES = [(2, 28), (3, 17), (4, 14), (5, 12)]
EPS32 = 2.0 ** -24


def bound(d, gates):
    return 2 * (2 * gates * d * EPS32)


def block_ranges(n):
    """Three blocks of consecutive qudits covering 0..n-1."""
    a = n // 3
    b = 2 * n // 3
    return [(0, a), (a, b), (b, n)]


def product_circuit(d, n, gates, seed):
    """Random benchmark-kind gates, each inside one block; returns the full
    circuit and the per-block circuits (block-local qudit indices)."""
    rng = np.random.default_rng([seed, d, n])
    blocks = block_ranges(n)
    full, local = [], [[] for _ in blocks]
    for _ in range(gates):
        bi = int(rng.integers(len(blocks)))
        lo, hi = blocks[bi]
        kind = W.RANDOM_KINDS[int(rng.integers(len(W.RANDOM_KINDS)))]
        op = W.random_gate(kind, d, hi - lo, rng)
        local[bi].append(op)
        full.append(W.Op(op.kind, tuple(q + lo for q in op.qudits), j=op.j, k=op.k, axis=op.axis,
                         theta=op.theta, param=op.param, power=op.power, matrix=op.matrix))
    return full, local, blocks


def inverse_ops(ops, d):
    """Each gate's inverse, in reverse order (gate kinds of the benchmark)."""
    inv = []
    for op in reversed(ops):
        if op.kind == "u":
            inv.append(W.Op("u", op.qudits, matrix=np.conj(np.asarray(op.matrix)).T))
        elif op.kind in ("rot", "crot"):
            inv.append(W.Op(op.kind, op.qudits, j=op.j, k=op.k, axis=op.axis, theta=-op.theta))
        elif op.kind in ("z", "x"):
            inv.append(W.Op(op.kind, op.qudits, power=d - op.power % d))
        elif op.kind == "sum":
            inv.extend(W.Op("sum", op.qudits) for _ in range(d - 1))
        else:
            raise ValueError(op.kind)
    return inv


def sample_indices(d, n, count, seed):
    N = d ** n
    rng = np.random.default_rng([seed, d, n])
    idx = rng.integers(0, N, size=count, dtype=np.int64)
    return np.unique(np.concatenate([idx, np.array([0, 1, N // 2, N - 2, N - 1], dtype=np.int64)]))


def expected_product(block_states, blocks, d, n, idx):
    out = np.ones(idx.shape, dtype=np.complex128)
    for psi_b, (lo, hi) in zip(block_states, blocks):
        digits = (idx // d ** (n - hi)) % d ** (hi - lo)
        out *= psi_b[digits]
    return out


# ---------------------------------------------------------------- host checks of the helpers (oracle only)
@pytest.mark.parametrize("d,n", [(2, 7), (3, 6), (5, 6)])
def test_product_helpers_on_oracle(orc, d, n):
    full, local, blocks = product_circuit(d, n, 40, seed=5)
    psi = orc.run(full, d, n)
    states = [orc.run(ops, d, hi - lo) for ops, (lo, hi) in zip(local, blocks)]
    idx = np.arange(d ** n, dtype=np.int64)
    np.testing.assert_allclose(psi, expected_product(states, blocks, d, n, idx), atol=1e-12)


@pytest.mark.parametrize("d,n", [(2, 6), (3, 4), (4, 3), (5, 3)])
def test_inverse_helper_on_oracle(orc, d, n):
    ops = W.random_circuit(d, n, 60)
    psi = orc.run(ops + inverse_ops(ops, d), d, n)
    e0 = np.zeros_like(psi)
    e0[0] = 1.0
    assert np.abs(psi - e0).max() < 1e-12


# ---------------------------------------------------------------- full sizes on the GPU
@pytest.mark.gpu
@pytest.mark.parametrize("d,n", SIZES)
def test_product_circuit_full_size_sampled(orc, d, n):
    import torch
    qf = gpu_lib()
    gates = 200
    full, local, blocks = product_circuit(d, n, gates, seed=11)
    states = [orc.run(ops, d, hi - lo) for ops, (lo, hi) in zip(local, blocks)]
    p = qf.program_from_ops(d, n, full, fuse=True)
    st = qf.State(d, n, "c64").set_basis(0)
    qf.qf_program_run(p, st.handle)
    torch.cuda.synchronize()
    idx = sample_indices(d, n, 4096, seed=3)
    got = st.tensor[torch.from_numpy(idx).to("cuda")].cpu().numpy().astype(np.complex128)
    want = expected_product(states, blocks, d, n, idx)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= bound(d, gates), rel
    norm = float((st.tensor.abs().double() ** 2).sum())
    assert abs(norm - 1.0) <= 2 * bound(d, gates)
    qf.qf_program_free(p)
    st.free()
    del st
    torch.cuda.empty_cache()


@pytest.mark.gpu
@pytest.mark.parametrize("d,n", SIZES)
def test_benchmark_sequence_full_size_roundtrip(d, n):
    import torch
    qf = gpu_lib()
    ops = W.random_circuit(d, n, 200)
    inv = inverse_ops(ops, d)
    p = qf.program_from_ops(d, n, ops, fuse=True)
    q = qf.program_from_ops(d, n, inv, fuse=True)
    st = qf.State(d, n, "c64").set_basis(0)
    qf.qf_program_run(p, st.handle)
    torch.cuda.synchronize()
    norm = float((st.tensor.abs().double() ** 2).sum())
    assert abs(norm - 1.0) <= 2 * bound(d, len(ops))
    qf.qf_program_run(q, st.handle)
    torch.cuda.synchronize()
    t = st.tensor
    err0 = float((t[0] - 1.0).abs())
    rest = float(t[1:].abs().max())
    assert err0 <= bound(d, len(ops) + len(inv)) and rest <= bound(d, len(ops) + len(inv)), (err0, rest)
    qf.qf_program_free(p)
    qf.qf_program_free(q)
    st.free()
    del st, t
    torch.cuda.empty_cache()
