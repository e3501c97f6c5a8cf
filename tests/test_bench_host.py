"""Host logic of bench.py's CPU-baseline leg: it times the oracle and states
the error of each GPU result it is handed.  Here the "GPU results" are the
oracle's own outputs (and one planted mistake), at small sizes, so the
comparison plumbing is checked without a GPU."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_cpu_baseline_error_statement(orc):
    import bench
    from paper_2409_17716_gb300 import workloads as W
    d, n = 3, 6
    exact = orc.run(W.random_circuit(d, n, bench.N_GATES), d, n)
    wrong = exact.copy()
    wrong[5] += 1e-3          # a planted mistake in the "complex64" result
    ad, an, L = 3, 4, 2
    aops, P = W.variational_ansatz(ad, an, L)
    theta = W.normal_angles(P, seed=4)
    w = [1.0] * an
    g = orc.grad_bruteforce(aops, ad, an, theta, w)
    l = orc.loss(orc.run(aops, ad, an, params=theta), ad, an, w)
    slots = [0, P - 1]
    circs, params = W.batch_circuits(count=3, seed=5, n_range=(2, 3), l_range=(1, 2))
    smp = []
    for c in circs:
        cw = [1.0] + [0.0] * (c.n - 1)
        used = sorted({op.param for op in c.ops if op.param >= 0})
        gg = orc.grad_bruteforce(c.ops, c.d, c.n, params, cw, slots=used)
        ll = orc.loss(orc.run(c.ops, c.d, c.n, params=params), c.d, c.n, cw)
        smp.append((c.ops, c.d, c.n, used, ll, gg, params))
    keep = {"forward": {"c64": wrong.astype(np.complex64), "c128": exact},
            "adjoint": {"d": ad, "n": an, "ops": aops, "theta": theta, "w": w, "P": P, "slots": slots,
                        "c128": (l, g)},
            "batched": {"dtype": "c64", "circuits": smp, "sample": "three small circuits"}}
    rec, err = bench.cpu_baseline(keep, size=(d, n))
    assert rec["kind"] == "oracle" and rec["cores"] >= 1 and rec["value"] > 0
    assert rec["one_thread"]["cores"] == 1
    assert err["forward_c128"]["max_abs"] == 0.0 and err["forward_c128"]["within"]
    assert 9e-4 < err["forward_c64"]["max_abs"] < 1.1e-3 and not err["forward_c64"]["within"]
    assert err["adjoint_c128"]["max_abs"] == 0.0 and err["adjoint_c128"]["loss_abs"] < 1e-14
    assert "adjoint_c64" not in err
    assert err["batched_c64"]["max_abs"] == 0.0 and err["batched_c64"]["loss_abs"] == 0.0
    assert orc.get_threads() == rec["cores"]
