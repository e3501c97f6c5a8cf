"""Helpers of the full-size parity tests (circuit builders and comparisons;
no gate arithmetic: the oracle and the CUDA path compute every state)."""
import numpy as np

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


def max_abs_diff_chunked(got, want, chunk=1 << 25):
    """max |got - want| over two equally long host arrays, in chunks (the
    full-size states hold up to 2.7e8 amplitudes)."""
    assert got.shape == want.shape
    m = 0.0
    for i in range(0, want.size, chunk):
        m = max(m, float(np.abs(got[i:i + chunk].astype(np.complex128) - want[i:i + chunk]).max()))
    return m
