"""Helpers shared by the GPU parity tests (imported only by tests marked gpu)."""
import numpy as np
import pytest


def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2409_17716_gb300 import build, qf
    build.build()
    qf.lib()
    return qf


def tol(dtype, gates=1):
    """Max-abs amplitude tolerances: complex128 1e-12; complex64 1e-5 after a
    200-gate circuit (about 5e-8 per gate for unit-norm states)."""
    if dtype == "c128":
        return 1e-12
    return 1e-6 if gates <= 20 else 1e-5


def upload(qf, psi, d, n, dtype):
    import torch
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    t = torch.from_numpy(np.ascontiguousarray(psi)).to(device="cuda", dtype=tdt)
    return qf.State(d, n, dtype, tensor=t)


def download(st):
    import torch
    torch.cuda.synchronize()
    return st.tensor.cpu().numpy().astype(np.complex128)
