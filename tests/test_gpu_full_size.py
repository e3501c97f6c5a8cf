"""Parity at the benchmark's full sizes (d=2 n=28, d=3 n=17, d=4 n=14,
d=5 n=12), complex64 and complex128, in the launch configuration the
benchmark times: fused programs with compiled tile passes and default
tiling, run through the C ABI.

* The benchmark's own 200-gate sequences against the complex128 oracle, every
  amplitude: max-abs error <= 1e-5 in complex64 and <= 1e-12 in complex128
  (the stated tolerances).  The oracle needs about a minute per size on the
  host cores.
* Product circuits.  Random gates of every kind the benchmark draws, each
  confined to one of three blocks of consecutive qudits, so the final state
  is the tensor product of three block states.  The oracle computes each
  block state; every sampled amplitude of the full state must equal the
  product of the three block amplitudes at the index's block digits (basis
  index i = sum_q i_q d^(n-1-q), qudit 0 most significant).
* The benchmark's own 200-gate sequences followed by their inverse (each
  gate's inverse, in reverse order) must return |0...0>, and the norm must
  be 1 after the forward half.

Tolerance of the product and round-trip checks: a complex64 d-term dot
product per gate and amplitude adds at most about 2 d 2^-24 relative error,
so after G gates the error vector's norm is below 2 G d 2^-24; the tests
allow twice that, for the round trip's distance from |0...0> and, relative
to the sampled amplitudes' norm, for the sampled amplitudes (rounding spreads
over the amplitudes like the state does, while a wrong gate, index or level
gives relative errors of order 1).
"""
import numpy as np
import pytest

from gpu_util import gpu_lib
from paper_2409_17716_gb300 import workloads as W

from fullsize_util import (SIZES, bound, expected_product, inverse_ops, max_abs_diff_chunked, product_circuit,
                           sample_indices)


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
def test_benchmark_sequence_full_size_vs_oracle(orc, d, n):
    """The timed 200-gate sequence, every amplitude against the oracle, in
    both precisions (the oracle's state is computed once per size)."""
    import torch
    qf = gpu_lib()
    ops = W.random_circuit(d, n, 200)
    want = orc.run(ops, d, n)
    p = qf.program_from_ops(d, n, ops, fuse=True)
    for dtype, atol in (("c64", 1e-5), ("c128", 1e-12)):
        st = qf.State(d, n, dtype).set_basis(0)
        qf.qf_program_run(p, st.handle)
        torch.cuda.synchronize()
        got = st.tensor.cpu().numpy()
        st.free()
        del st
        torch.cuda.empty_cache()
        err = max_abs_diff_chunked(got, want)
        print("benchmark sequence d=%d n=%d %s: max-abs error vs oracle %.3g" % (d, n, dtype, err))
        assert err <= atol, (dtype, err)
        del got
    qf.qf_program_free(p)


@pytest.mark.gpu
@pytest.mark.parametrize("d,n", SIZES)
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_product_circuit_full_size_sampled(orc, d, n, dtype):
    import torch
    qf = gpu_lib()
    gates = 200
    full, local, blocks = product_circuit(d, n, gates, seed=11)
    states = [orc.run(ops, d, hi - lo) for ops, (lo, hi) in zip(local, blocks)]
    p = qf.program_from_ops(d, n, full, fuse=True)
    st = qf.State(d, n, dtype).set_basis(0)
    qf.qf_program_run(p, st.handle)
    torch.cuda.synchronize()
    idx = sample_indices(d, n, 4096, seed=3)
    got = st.tensor[torch.from_numpy(idx).to("cuda")].cpu().numpy().astype(np.complex128)
    want = expected_product(states, blocks, d, n, idx)
    if dtype == "c64":
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert rel <= bound(d, gates), rel
        norm = float((st.tensor.abs().double() ** 2).sum())
        assert abs(norm - 1.0) <= 2 * bound(d, gates)
    else:
        assert np.abs(got - want).max() <= 1e-12
        assert abs(st.expect_number()[n] - 1.0) <= 1e-12
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
