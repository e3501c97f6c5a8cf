"""qf_program_run_expect: <N_q> and the norm reduced inside the program's
last pass (compiled complex64 tile pass), against qf_program_run followed by
the separate reduction, and against the oracle on small states; the
fallbacks (complex128, a last pass that is not a tile pass) give the same
values; a 32-qubit state (33 outputs: two per lane of a warp)."""
import numpy as np
import pytest

from gpu_util import gpu_lib
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _both(qf, d, n, ops, dtype):
    import torch
    st = qf.State(d, n, dtype).set_basis(0)
    p = qf.program_from_ops(d, n, ops)
    out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    qf.qf_program_run_expect(p, st.handle, out.data_ptr())
    fused = out.cpu().numpy().copy()
    st.set_basis(0)
    qf.qf_program_run(p, st.handle)
    sep = st.expect_number()
    psi = st.tensor.cpu().numpy().astype(np.complex128)
    qf.qf_program_free(p)
    st.free()
    return fused, sep, psi


@pytest.mark.parametrize("d,n", [(2, 14), (3, 9), (4, 7), (5, 6), (7, 4), (3, 13)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_fused_matches_separate_and_oracle(orc, d, n, dtype):
    qf = gpu_lib()
    ops = [W.Op("h", (q,)) for q in range(n)] + W.random_circuit(d, n, 120, seed=d * 31 + n)
    fused, sep, psi = _both(qf, d, n, ops, dtype)
    want = orc.expect_number(orc.run(ops, d, n), d, n)
    tol = 1e-12 if dtype == "c128" else 1e-6 * n * d
    assert np.abs(fused[:n] - want).max() <= tol
    assert abs(fused[n] - 1.0) <= (1e-12 if dtype == "c128" else 1e-5)
    assert np.abs(fused - sep).max() <= (1e-12 if dtype == "c128" else 2e-6 * n * d)


def test_last_pass_strided_falls_back(orc):
    qf = gpu_lib()
    d, n = 3, 10
    # a lone wide-stride gate at the end runs through the strided kernel
    ops = W.random_circuit(d, n, 60, seed=4) + [W.Op("rot", (0,), j=0, k=2, axis="x", theta=0.8)]
    fused, sep, _ = _both(qf, d, n, ops, "c64")
    want = orc.expect_number(orc.run(ops, d, n), d, n)
    assert np.abs(fused[:n] - want).max() <= 1e-6 * n * d
    assert np.abs(fused - sep).max() <= 2e-6 * n * d


def test_thirty_two_qubits():
    """33 outputs: lane c of a warp holds outputs c and c + 32."""
    import torch
    qf = gpu_lib()
    d, n = 2, 32
    free, _ = torch.cuda.mem_get_info()
    assert free > 40e9
    rng = np.random.default_rng(3)
    ops = [W.Op("h", (q,)) for q in range(0, n, 3)]
    ops += [W.Op("rot", (int(q),), j=0, k=1, axis="y", theta=float(rng.uniform(0, 6))) for q in rng.integers(0, n, 12)]
    ops += [W.Op("sum", (q, q + 1)) for q in range(0, n - 1, 7)]
    fused, sep, _ = _both(qf, d, n, ops, "c64")
    assert fused.shape == (n + 1,)
    assert np.abs(fused - sep).max() <= 2e-6 * n
    assert abs(fused[n] - 1.0) <= 1e-5
    torch.cuda.empty_cache()
