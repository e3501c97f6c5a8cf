"""C ABI checks that need no GPU: the library loads, exports every entry point
include/qf.h declares, rejects invalid arguments on the host before touching
CUDA, and plans fused passes (host-only planner)."""
import os
import re

import pytest

from paper_2409_17716_gb300 import build as gpu_build
from paper_2409_17716_gb300 import qf, workloads

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qf.h")


@pytest.fixture(scope="module")
def L():
    gpu_build.build()
    return qf.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["qf_state_init", "qf_apply_gate", "qf_apply_rot", "qf_apply_sum", "qf_expect", "qf_program_run"]:
        assert must in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_every_declared_symbol_is_bound():
    assert set(declared_functions()) <= set(qf._PROTOS), set(declared_functions()) - set(qf._PROTOS)


def test_invalid_arguments_rejected_on_host(L):
    for d, n in [(1, 3), (17, 2), (3, 0), (3, 63)]:
        with pytest.raises(qf.QFError) as ei:
            qf.qf_state_init(d, n, qf.QF_C64, stream=0)
        assert ei.value.status == qf.QF_ERR_ARG
    with pytest.raises(qf.QFError) as ei:
        qf.qf_program_create(1, 4)
    assert ei.value.status == qf.QF_ERR_ARG
    assert qf.qf_expect_size(3, 5, qf.QF_OBS_NUMBER_ALL) == 6
    assert qf.qf_expect_size(3, 5, qf.QF_OBS_MARGINAL) == 3
    assert qf.qf_expect_size(3, 5, 99) == -1


def test_program_validation_on_host(L):
    p = qf.qf_program_create(3, 4)
    try:
        bad = [lambda: qf.qf_program_add_rot(p, 4, 0, 1, "x"),       # qudit out of range
               lambda: qf.qf_program_add_rot(p, 0, 1, 1, "y"),       # j == k
               lambda: qf.qf_program_add_rot(p, 0, 0, 3, "x"),       # k >= d
               lambda: qf.qf_program_add_rot(p, 0, 0, 1, "q"),       # axis
               lambda: qf.qf_program_add_rot(p, 0, 3, 0, "g"),       # Gell-Mann j > d-1
               lambda: qf.qf_program_add_sum(p, 2, 2),               # c == t
               lambda: qf.qf_program_add_crot(p, 1, 1, 0, 1, "y"),
               lambda: qf.qf_program_add_gate(p, [0, 0], [[1]])]
        for f in bad:
            with pytest.raises(qf.QFError) as ei:
                f()
            assert ei.value.status == qf.QF_ERR_ARG
        with pytest.raises(qf.QFError) as ei:
            import numpy as np
            qf.qf_program_add_gate(p, [0, 1, 2, 3], np.eye(81))       # d^k = 81 > 64
        assert ei.value.status == qf.QF_ERR_UNSUPPORTED
        assert qf.qf_program_info(p) == (0, 0)
        qf.qf_program_add_rot(p, 0, 0, 1, "y", param_slot=7)
        assert qf.qf_program_info(p) == (1, 8)
    finally:
        qf.qf_program_free(p)


def test_planner_fuses_and_respects_limits(L):
    d, n = 3, 17
    ops = workloads.random_circuit(d, n, 200)
    pf = qf.program_from_ops(d, n, ops, fuse=True)
    pu = qf.program_from_ops(d, n, ops, fuse=False)
    try:
        fused = qf.qf_program_plan(pf, qf.QF_C64)
        unfused = qf.qf_program_plan(pu, qf.QF_C64)
        assert unfused[0] == 200 and unfused[2] == 1
        assert fused[0] < 100, fused          # several gates per pass
        assert fused[2] <= 96
    finally:
        qf.qf_program_free(pf)
        qf.qf_program_free(pu)


def test_planner_small_state_single_tile(L):
    d, n = 3, 6
    ops = workloads.layered_circuit(d, n, layers=2)
    p = qf.program_from_ops(d, n, ops, fuse=True)
    try:
        passes, strided, max_ops = qf.qf_program_plan(p, qf.QF_C128)
        assert strided == 0 and passes == 1   # 729 amplitudes fit one tile
    finally:
        qf.qf_program_free(p)


def test_program_controls_validation_on_host(L):
    """Tiling, stage-slot and multi-controlled-gate arguments are checked on
    the host; a rejected call records nothing."""
    import numpy as np
    p = qf.qf_program_create(3, 4)
    try:
        bad = [lambda: qf.qf_program_set_tiling(p, -1, 0, 0),
               lambda: qf.qf_program_set_stage_slots(p, 7),
               lambda: qf.qf_program_add_mcx(p, [1, 2], 2),         # control == target
               lambda: qf.qf_program_add_mcx(p, [1, 1], 2),         # repeated control
               lambda: qf.qf_program_add_mcx(p, [1, 4], 2),         # qudit out of range
               lambda: qf.qf_program_add_mcx(p, [], 2),             # no control
               lambda: qf.qf_program_add_mcu(p, [0], [3], 1, np.eye(3)),   # control level >= d
               lambda: qf.qf_program_create_dims([2, 1, 3])]
        for f in bad:
            with pytest.raises(qf.QFError) as ei:
                f()
            assert ei.value.status == qf.QF_ERR_ARG
        assert qf.qf_program_info(p) == (0, 0)
        qf.qf_program_set_tiling(p, 6, 2, 10)
        qf.qf_program_set_stage_slots(p, 6)
        qf.qf_program_add_mcx(p, [0, 1], 3)
        assert qf.qf_program_info(p) == (1, 0)
    finally:
        qf.qf_program_free(p)
