"""The CUDA source a program's compiled tile passes are built from compiles
with NVRTC for sm_103a (host only, no GPU): every gate kind, controls inside
and outside a register stage, shared-memory SWAP and multi-qudit gates,
complex64 and complex128, default and overridden stage slots."""
import ctypes
import math
import os

import numpy as np
import pytest

from paper_2409_17716_gb300 import qf, workloads as W


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", os.path.join("/usr/local/cuda/lib64", "libnvrtc.so")):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC not available")


def _compile(L, src):
    prog = ctypes.c_void_p()
    assert L.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"t.cu", 0, None, None) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"-default-device"]
    rc = L.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    L.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(max(n.value, 1))
    L.nvrtcGetProgramLog(prog, log)
    L.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace")


def _units(p, dtype):
    src = qf.qf_program_jit_source(p, dtype)
    return [u for u in src.split("// ---- translation unit\n") if u.strip()]


CASES = [
    ("d3 random", 3, 9, lambda: W.random_circuit(3, 9, 40), qf.QF_C64, 0),
    ("d2 random c128", 2, 12, lambda: W.random_circuit(2, 12, 40), qf.QF_C128, 0),
    ("d5 random", 5, 5, lambda: W.random_circuit(5, 5, 30), qf.QF_C64, 0),
    ("d4 slots 1", 4, 6, lambda: W.random_circuit(4, 6, 30), qf.QF_C64, 1),
]


@pytest.mark.parametrize("name,d,n,mk,dtype,slots", CASES, ids=[c[0] for c in CASES])
def test_generated_passes_compile(name, d, n, mk, dtype, slots):
    L = _nvrtc()
    p = qf.program_from_ops(d, n, mk())
    qf.qf_program_set_stage_slots(p, slots)
    units = _units(p, dtype)
    assert units
    for u in units[:2]:
        rc, log = _compile(L, u)
        assert rc == 0, log[:2000]
    qf.qf_program_free(p)


def test_generated_special_ops_compile():
    """SWAP and a two-qudit dense gate (shared-memory ops), controlled
    rotations with the control outside the stage, a multi-controlled gate
    (its own pass, no compiled source)."""
    L = _nvrtc()
    d, n = 3, 7
    rng = np.random.default_rng(1)
    ops = [W.Op("h", (q,)) for q in range(n)]
    ops += [W.Op("swap", (1, 5)), W.Op("u", (2, 6), matrix=W.haar_unitary(9, rng)),
            W.Op("crot", (0, 6), j=0, k=2, axis="x", theta=0.3), W.Op("crot", (6, 0), j=1, k=2, axis="z", theta=0.5),
            W.Op("sum", (5, 6)), W.Op("sum", (6, 1)), W.Op("rot", (3,), j=2, axis="g", theta=0.2),
            W.Op("mcx", (0, 1, 2)), W.Op("z", (4,), power=2), W.Op("x", (4,), power=1)]
    p = qf.program_from_ops(d, n, ops)
    units = _units(p, qf.QF_C64)
    src = "".join(units)
    assert "const int e2 = e +" in src and "offs[" in src     # SWAP and dense k-qudit code present
    assert "const int tp = (int)(base & 1);" in src           # odd d, complex64: padded tile layout
    for u in units:
        rc, log = _compile(L, u)
        assert rc == 0, log[:2000]
    qf.qf_program_free(p)


@pytest.mark.parametrize("d,n,dtype", [(3, 8, qf.QF_C64), (2, 10, qf.QF_C128), (5, 4, qf.QF_C64)])
def test_generated_adjoint_passes_compile(d, n, dtype):
    """Reverse passes of the adjoint sweep: psi and lambda register blocks,
    gradient terms of rotations and controlled rotations (controls inside
    and outside a stage), shared-memory SWAP on both tiles."""
    L = _nvrtc()
    ops, P = W.variational_ansatz(d, n, 2)
    ops = ops + [W.Op("crot", (0, n - 1), j=0, k=1, axis="y", param=0),
                 W.Op("crot", (n - 1, 1), j=0, k=1, axis="z", param=1), W.Op("swap", (1, 2)),
                 W.Op("rot", (2,), j=d - 1, axis="g", param=2)]
    p = qf.program_from_ops(d, n, ops)
    src = qf.qf_program_jit_source(p, dtype, adjoint=True)
    units = [u for u in src.split("// ---- translation unit\n") if u.strip()]
    assert units and "A.rows[" in src and "ltile" in src
    for u in sorted(units, key=len)[-2:]:
        rc, log = _compile(L, u)
        assert rc == 0, log[:2000]
    qf.qf_program_free(p)


def _tile_sizes(src):
    import re
    return sorted({int(x) for x in re.findall(r"// tile of (\d+) amplitudes", src)} |
                  {int(x) for x in re.findall(r"ltile = tile \+ (\d+);", src)})


def test_tiling_defaults_and_overrides():
    """Planner tiles as the generated source shows them: forward qubit passes
    in complex64 on 4096-amplitude tiles (the adjoint keeps 8192, complex128
    4096), d=4 forward passes on 128-thread CTAs, and tile overrides up to the
    160 KiB limit (larger requests clamp to it)."""
    ops2 = W.random_circuit(2, 16, 60)
    p = qf.program_from_ops(2, 16, ops2)
    assert _tile_sizes(qf.qf_program_jit_source(p, qf.QF_C64)) == [4096]
    assert _tile_sizes(qf.qf_program_jit_source(p, qf.QF_C64, adjoint=True)) == [8192]
    assert _tile_sizes(qf.qf_program_jit_source(p, qf.QF_C128)) == [4096]
    qf.qf_program_set_tiling(p, 15, 0, 0)   # 256 KiB asked: clamps to 2^14 amplitudes (128 KiB)
    assert _tile_sizes(qf.qf_program_jit_source(p, qf.QF_C64)) == [16384]
    qf.qf_program_free(p)
    p = qf.program_from_ops(4, 8, W.random_circuit(4, 8, 40))
    src = qf.qf_program_jit_source(p, qf.QF_C64)
    assert _tile_sizes(src) == [4096] and "__launch_bounds__(128)" in src and "__launch_bounds__(256)" not in src
    qf.qf_program_free(p)


@pytest.mark.parametrize("d,n,tile,run", [(3, 11, 9, 0), (5, 8, 6, 2), (2, 16, 14, 4)])
def test_large_tile_passes_compile(d, n, tile, run):
    L = _nvrtc()
    p = qf.program_from_ops(d, n, W.random_circuit(d, n, 60))
    qf.qf_program_set_tiling(p, tile, run, 0)
    units = _units(p, qf.QF_C64)
    assert _tile_sizes("".join(units)) == [d ** tile]
    rc, log = _compile(L, max(units, key=len))
    assert rc == 0, log[:2000]
    qf.qf_program_free(p)


def _compile_v(L, src):
    prog = ctypes.c_void_p()
    assert L.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"t.cu", 0, None, None) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"-default-device", b"--ptxas-options=-v"]
    rc = L.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    L.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(max(n.value, 1))
    L.nvrtcGetProgramLog(prog, log)
    L.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace")


@pytest.mark.parametrize("d,n", [(2, 28), (3, 17), (4, 14), (5, 12)])
def test_benchmark_passes_compile_without_spills(d, n):
    """Every compiled pass of the benchmark's random 200-gate programs
    compiles for sm_103a without register spills beyond a few words
    (ptxas report), at the default stage slots and tiling.  A capped
    register budget spills hundreds of bytes per pass; ptxas alone may still
    park up to 16 bytes of loop-invariant values on the stack."""
    import re
    from concurrent.futures import ThreadPoolExecutor
    L = _nvrtc()
    p = qf.program_from_ops(d, n, W.random_circuit(d, n, 200))
    units = _units(p, qf.QF_C64)
    qf.qf_program_free(p)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda u: _compile_v(L, u), units))
    for rc, log in results:
        assert rc == 0, log[:2000]
        spills = [int(x) for x in re.findall(r"(\d+) bytes spill stores", log)]
        assert spills and max(spills) <= 16, log[-600:]


def test_direct_stages():
    """Forward passes whose first (complex64, odd d) or last register stage
    holds only active qudits read or write HBM directly from the stage's
    registers: the source says so in its stage summary, such a pass has no
    tile copy on that side, and the global offsets of a direct stage's
    registers are the active strides' digit sums.  The pass that reduces
    <N_q> keeps its shared-memory tile; complex128 passes store directly
    but load through shared memory."""
    import re
    L = _nvrtc()
    d, n = 3, 17
    p = qf.program_from_ops(d, n, W.random_circuit(d, n, 200))
    units = _units(p, qf.QF_C64)
    tags = [re.search(r"// register stages: ([^\n]*)", u).group(1) for u in units]
    assert any("first from HBM" in t for t in tags) and any("last to HBM" in t for t in tags)
    assert "HBM" not in tags[-1]   # the reducing pass
    for u, t in zip(units, tags):
        if "first from HBM" in t:
            assert "for (; t <" in u and "qj_cp2(" not in u.split("for (; t <")[1]
            # run-number digit 0 first, as the offA table composes them
            strides = [int(x) for x in re.findall(r"o \+= \(long long\)\(rem % 3\) \* (\d+)LL", u)]
            seg = int(re.search(r"const int gab = b / (\d+);", u).group(1))
            first = u.split("for (int blk = tid; blk <")[1]
            ins = [int(x) for x in re.findall(r"const int q = b / (\d+); b = q \*", first.split("C v0")[0])]
            offs = [int(x) for x in re.findall(r"C v\d+ = gq\[(\d+)LL\];", first)]
            # slot strides, most significant first, as run-number digits
            digs = sorted((round(math.log(s // seg, 3)) for s in ins), reverse=True)
            want = []
            for r in range(d ** len(digs)):
                g = 0
                for i, dg in enumerate(digs):
                    g += ((r // d ** (len(digs) - 1 - i)) % d) * strides[dg]
                want.append(g)
            assert offs == want, (offs, want)
        if "last to HBM" in t:
            assert "qj_st2(A.psi" not in u and "A.psi[g" not in u
    for u in units[:3]:
        rc, log = _compile(L, u)
        assert rc == 0, log[:2000]
    c128 = _units(p, qf.QF_C128)
    ct = [re.search(r"// register stages: ([^\n]*)", u).group(1) for u in c128]
    assert any("last to HBM" in t for t in ct) and not any("first from HBM" in t for t in ct)
    rc, log = _compile(L, next(u for u, t in zip(c128, ct) if "last to HBM" in t))
    assert rc == 0, log[:2000]
    qf.qf_program_free(p)


@pytest.mark.parametrize("d,n,dtype,adjoint", [(3, 12, qf.QF_C64, False), (5, 8, qf.QF_C64, True), (7, 6, qf.QF_C64, False),
                                               (4, 8, qf.QF_C128, False), (3, 10, qf.QF_C128, True)])
def test_direct_stage_variants_compile(d, n, dtype, adjoint):
    """Direct stages and the L2 prefetch in other shapes: odd and even d,
    d = 7, forward and adjoint, complex64 and complex128 (double-float), with
    shared-memory SWAPs between register stages; every unit with a direct
    stage compiles.  The prefetch appears only in complex64 forward passes at
    odd d whose runs are at least 128 bytes."""
    import re
    L = _nvrtc()
    ops = W.random_circuit(d, n, 50) + [W.Op("swap", (0, n - 1))] + W.random_circuit(d, n, 30, seed=7)
    if adjoint:
        ops, _ = W.variational_ansatz(d, n, 2, entangler="chain")
    p = qf.program_from_ops(d, n, ops)
    src = qf.qf_program_jit_source(p, dtype, adjoint=adjoint)
    units = [u for u in src.split("// ---- translation unit\n") if u.strip()]
    direct = [u for u in units if "HBM" in re.search(r"// register stages: ([^\n]*)", u).group(1)]
    assert direct
    for u in direct[:3]:
        rc, log = _compile(L, u)
        assert rc == 0, log[:2000]
        if "first from HBM" in u:
            assert dtype == qf.QF_C64 and d % 2 == 1
    for u in units:
        if "prefetch.L2" in u:
            seg = int(re.search(r"tile of (\d+)", u).group(1)) // int(re.search(r"for \(int a = tid; a < (\d+);", u).group(1))
            assert dtype == qf.QF_C64 and not adjoint and d % 2 == 1 and seg * 8 >= 128
    qf.qf_program_free(p)
