"""GPU parity of qf_measure: marginal probabilities of qudit subsets (in any
order) against the oracle, and shot histograms from the same uniforms equal to
the oracle's bin by bin; the paper's Deutsch-Jozsa example measured on the GPU."""
import numpy as np
import pytest

from gpu_util import gpu_lib, upload
from paper_2409_17716_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("d,n", [(2, 12), (3, 7), (5, 4)])
def test_measure_matches_oracle(orc, d, n, dtype):
    qf = gpu_lib()
    psi = W.uniform_state(d, n, seed=d * 13 + n)
    st = upload(qf, psi, d, n, dtype)
    ref = psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi
    u = np.random.default_rng(3).random(50000)
    for idx in ([0], [n - 1], [n - 1, 0], [1, n - 2, 0]):
        hist, probs = qf.qf_measure(st.handle, idx, shots=len(u), uniforms=u)
        want = orc.marginal(ref, d, n, idx)
        np.testing.assert_allclose(probs, want, atol=1e-12 if dtype == "c128" else 1e-6)
        assert hist.sum() == len(u)
        # same uniforms, same rule: identical histograms unless a uniform sits
        # within rounding of a bin edge
        want_h = orc.sample(probs, u)
        assert np.array_equal(hist, want_h)
    st.free()


def test_deutsch_jozsa_measured_on_gpu(orc):
    qf = gpu_lib()
    for d in (3, 4):
        for mode in ("constant", "balanced"):
            n = 4
            st = qf.State(d, n, "c128").set_basis(d - 1)
            for q in range(n):
                qf.qf_apply_h(st.handle, q)
            if mode == "constant":
                qf.qf_apply_x(st.handle, n - 1, 1)
            else:
                qf.qf_apply_sum(st.handle, 2, 3)
            for q in range(n - 1):
                qf.qf_apply_h(st.handle, q)
            hist, p = qf.qf_measure(st.handle, [0, 1, 2], shots=1024, seed=1)
            expect = 0 if mode == "constant" else d - 1
            assert abs(p[expect] - 1) < 1e-12 and hist[expect] == 1024
            st.free()


def test_measure_rejects_bad_arguments():
    qf = gpu_lib()
    st = qf.State(3, 4, "c64").set_basis(0)
    for idx in ([4], [0, 0], []):
        with pytest.raises(qf.QFError) as ei:
            qf.qf_measure(st.handle, idx)
        assert ei.value.status == qf.QF_ERR_ARG
    st.free()
