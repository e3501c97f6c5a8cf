"""Python face of the CPU oracle.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
CPU-baseline leg of the benchmark.  It wraps ``qf_oracle.c`` (complex128,
explicit loops, gates built from the paper's Appendix B definitions) and adds
the circuit runner and the two gradient references:

* ``grad_bruteforce`` -- for every parameter, the circuit is re-run with each
  gate that uses it replaced by dU/dtheta (product rule over occurrences),
  giving |d_p psi>, and g_p = 2 Re <psi| O |d_p psi> for the diagonal
  observable O = sum_q w_q N_q.  Independent of any adjoint recursion.
* ``grad_fd`` -- central finite differences of the loss.

Ops are read by attribute (kind, qudits, j, k, axis, theta, param, power,
matrix); the oracle does not import the input generator.

Wherever a function takes ``d`` it also accepts a sequence of per-qudit
dimensions (mixed-dimension registers, section "Code style":
``Circuit(dim=[2,3,4])``); the basis index is then mixed-radix with qudit 0
most significant.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_LIB = None
_c = ctypes
_cp = _c.c_void_p


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = _c.CDLL(path)
        L.or_apply.argtypes = [_cp, _c.c_int, _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _cp]
        L.or_apply.restype = _c.c_int
        L.or_apply_dims.argtypes = [_cp, _c.POINTER(_c.c_int), _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _cp]
        L.or_apply_dims.restype = _c.c_int
        for name in ("or_gate_crot2", "or_gate_crot2_deriv"):
            f = getattr(L, name)
            f.argtypes = [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_char, _cp]
            f.restype = _c.c_int
        L.or_gate_sum2.argtypes = [_c.c_int, _c.c_int, _cp]
        L.or_gate_mcx.argtypes = [_c.POINTER(_c.c_int), _c.c_int, _c.c_int, _c.c_int, _cp]
        L.or_gate_mcx.restype = _c.c_int
        L.or_gate_mcu.argtypes = [_c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.c_int, _c.c_int, _cp, _cp]
        L.or_gate_mcu.restype = _c.c_int
        L.or_expect_number_dims.argtypes = [_cp, _c.POINTER(_c.c_int), _c.c_int, _cp]
        L.or_expect_obs_dims.argtypes = [_cp, _c.POINTER(_c.c_int), _c.c_int, _c.c_int, _cp, _cp, _cp]
        L.or_marginal_dims.argtypes = [_cp, _c.POINTER(_c.c_int), _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _cp]
        for name in ("or_gate_rot", "or_gate_rot_deriv", "or_gate_crot", "or_gate_crot_deriv"):
            f = getattr(L, name)
            f.argtypes = [_c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_char, _cp]
            f.restype = _c.c_int
        L.or_generator.argtypes = [_c.c_int, _c.c_int, _c.c_int, _c.c_char, _cp]
        L.or_generator.restype = _c.c_int
        L.or_gate_identity.argtypes = [_c.c_int, _cp]
        L.or_gate_fourier.argtypes = [_c.c_int, _cp]
        L.or_gate_shift.argtypes = [_c.c_int, _c.c_int, _cp]
        L.or_gate_clock.argtypes = [_c.c_int, _c.c_int, _cp]
        L.or_gate_sum.argtypes = [_c.c_int, _cp]
        L.or_gate_swap.argtypes = [_c.c_int, _cp]
        L.or_norm2.argtypes = [_cp, _c.c_longlong]
        L.or_norm2.restype = _c.c_double
        L.or_expect_number.argtypes = [_cp, _c.c_int, _c.c_int, _cp]
        L.or_expect_obs.argtypes = [_cp, _c.c_int, _c.c_int, _c.c_int, _cp, _cp, _cp]
        L.or_marginal.argtypes = [_cp, _c.c_int, _c.c_int, _c.POINTER(_c.c_int), _c.c_int, _cp]
        L.or_inner.argtypes = [_cp, _cp, _c.c_longlong, _cp, _cp]
        L.or_basis_state.argtypes = [_cp, _c.c_longlong, _c.c_longlong]
        L.or_set_threads.argtypes = [_c.c_int]
        L.or_get_threads.restype = _c.c_int
        _LIB = L
    return _LIB


def set_threads(t: int) -> None:
    """Host threads of the oracle's OpenMP loops (results do not depend on it)."""
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_cp)


def _cmat(m: int) -> np.ndarray:
    return np.zeros((m, m), dtype=np.complex128)


def dims_of(d, n: int):
    """Per-qudit dimensions: d repeated n times, or the sequence d itself."""
    if isinstance(d, (int, np.integer)):
        return [int(d)] * n
    dims = [int(x) for x in d]
    if len(dims) != n:
        raise ValueError("dims has %d entries for %d qudits" % (len(dims), n))
    return dims


def _ivec(v):
    return (_c.c_int * len(v))(*[int(x) for x in v])


def _chk(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle: invalid arguments to " + what)


# ---------------------------------------------------------------- gate builders
def identity(d):
    U = _cmat(d); lib().or_gate_identity(d, _ptr(U)); return U


def fourier(d):
    U = _cmat(d); lib().or_gate_fourier(d, _ptr(U)); return U


def shift(d, s=1):
    U = _cmat(d); lib().or_gate_shift(d, int(s), _ptr(U)); return U


def clock(d, p=1):
    U = _cmat(d); lib().or_gate_clock(d, int(p), _ptr(U)); return U


def generator(d, j, k, axis):
    S = _cmat(d); _chk(lib().or_generator(d, j, k, axis.encode(), _ptr(S)), "generator"); return S


def rot(d, j, k, theta, axis):
    U = _cmat(d); _chk(lib().or_gate_rot(d, j, k, float(theta), axis.encode(), _ptr(U)), "rot"); return U


def rot_deriv(d, j, k, theta, axis):
    U = _cmat(d); _chk(lib().or_gate_rot_deriv(d, j, k, float(theta), axis.encode(), _ptr(U)), "rot_deriv"); return U


def sum_gate(d, dt=None):
    """SUM with control dimension d and target dimension dt (default d)."""
    dt = d if dt is None else dt
    U = _cmat(d * dt); lib().or_gate_sum2(d, dt, _ptr(U)); return U


def swap_gate(d):
    U = _cmat(d * d); lib().or_gate_swap(d, _ptr(U)); return U


def crot(d, j, k, theta, axis, dt=None):
    """Controlled rotation, control dimension d, target dimension dt (default d)."""
    dt = d if dt is None else dt
    U = _cmat(d * dt)
    _chk(lib().or_gate_crot2(d, dt, j, k, float(theta), axis.encode(), _ptr(U)), "crot")
    return U


def crot_deriv(d, j, k, theta, axis, dt=None):
    dt = d if dt is None else dt
    U = _cmat(d * dt)
    _chk(lib().or_gate_crot2_deriv(d, dt, j, k, float(theta), axis.encode(), _ptr(U)), "crot_deriv")
    return U


def mcx_gate(dcs, dt, s=1):
    """Multi-controlled X^s: target += s * (product of the control levels)."""
    C = int(np.prod(dcs))
    U = _cmat(C * dt)
    _chk(lib().or_gate_mcx(_ivec(dcs), len(dcs), dt, int(s), _ptr(U)), "mcx")
    return U


def mcu_gate(dcs, levels, dt, V):
    """V on the target when control i is at levels[i] for every i."""
    C = int(np.prod(dcs))
    U = _cmat(C * dt)
    V = np.ascontiguousarray(V, dtype=np.complex128)
    assert V.shape == (dt, dt)
    _chk(lib().or_gate_mcu(_ivec(dcs), _ivec(levels), len(dcs), dt, _ptr(V), _ptr(U)), "mcu")
    return U


# ---------------------------------------------------------------- states
def basis(d, n, index=0):
    psi = np.zeros(int(np.prod(dims_of(d, n), dtype=np.int64)), dtype=np.complex128)
    lib().or_basis_state(_ptr(psi), psi.size, int(index))
    return psi


def apply(psi: np.ndarray, d, n: int, targets, U: np.ndarray) -> np.ndarray:
    """In place: psi <- (U on targets) psi."""
    dims = dims_of(d, n)
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == int(np.prod(dims, dtype=np.int64))
    U = np.ascontiguousarray(U, dtype=np.complex128)
    if any(not 0 <= int(t) < n for t in targets):
        raise ValueError("oracle: target qudit out of range")
    K = int(np.prod([dims[t] for t in targets]))
    assert U.shape == (K, K)
    _chk(lib().or_apply_dims(_ptr(psi), _ivec(dims), n, _ivec(targets), len(targets), _ptr(U)), "apply")
    return psi


def norm2(psi):
    return float(lib().or_norm2(_ptr(np.ascontiguousarray(psi)), psi.size))


def expect_number(psi, d, n):
    out = np.zeros(n)
    lib().or_expect_number_dims(_ptr(np.ascontiguousarray(psi)), _ivec(dims_of(d, n)), n, _ptr(out))
    return out


def expect_obs(psi, d, n, q, O):
    re, im = np.zeros(1), np.zeros(1)
    O = np.ascontiguousarray(O, dtype=np.complex128)
    lib().or_expect_obs_dims(_ptr(np.ascontiguousarray(psi)), _ivec(dims_of(d, n)), n, q, _ptr(O), _ptr(re), _ptr(im))
    return complex(re[0], im[0])


def marginal(psi, d, n, idx):
    dims = dims_of(d, n)
    out = np.zeros(int(np.prod([dims[q] for q in idx])))
    lib().or_marginal_dims(_ptr(np.ascontiguousarray(psi)), _ivec(dims), n, _ivec(idx), len(idx), _ptr(out))
    return out


def inner(a, b):
    re, im = np.zeros(1), np.zeros(1)
    lib().or_inner(_ptr(np.ascontiguousarray(a)), _ptr(np.ascontiguousarray(b)), a.size, _ptr(re), _ptr(im))
    return complex(re[0], im[0])


# ---------------------------------------------------------------- circuits
def op_matrix(op, d, params: Optional[Sequence[float]] = None, deriv: bool = False):
    """(targets, U) for one op; with deriv=True, (targets, dU/dtheta).  d is
    the register's dimension or its per-qudit dimensions."""
    k = op.kind
    if deriv and k not in ("rot", "crot"):
        raise ValueError("op %s has no angle" % k)
    if isinstance(d, (int, np.integer)):
        dq = lambda q: int(d)
    else:
        dq = lambda q: int(d[q])
    t0 = dq(op.qudits[0])
    if k == "h":
        return op.qudits, fourier(t0)
    if k == "x":
        return op.qudits, shift(t0, op.power)
    if k == "z":
        return op.qudits, clock(t0, op.power)
    if k == "rot":
        th = op.angle(params)
        f = rot_deriv if deriv else rot
        return op.qudits, f(t0, op.j, op.k, th, op.axis)
    if k == "crot":
        th = op.angle(params)
        f = crot_deriv if deriv else crot
        return op.qudits, f(t0, op.j, op.k, th, op.axis, dt=dq(op.qudits[1]))
    if k == "sum":
        return op.qudits, sum_gate(t0, dq(op.qudits[1]))
    if k == "swap":
        if dq(op.qudits[1]) != t0:
            raise ValueError("SWAP needs two qudits of the same dimension")
        return op.qudits, swap_gate(t0)
    if k == "u":
        return op.qudits, np.asarray(op.matrix, dtype=np.complex128)
    if k == "mcx":
        return op.qudits, mcx_gate([dq(q) for q in op.qudits[:-1]], dq(op.qudits[-1]), op.power)
    if k == "mcu":
        return op.qudits, mcu_gate([dq(q) for q in op.qudits[:-1]], op.levels, dq(op.qudits[-1]), op.matrix)
    raise ValueError("unknown op kind " + k)


def run(ops, d, n: int, psi: Optional[np.ndarray] = None, params=None) -> np.ndarray:
    """Applies ops in order to psi (default |0...0>); returns the final state
    (psi is copied, not modified)."""
    out = basis(d, n, 0) if psi is None else np.array(psi, dtype=np.complex128, copy=True)
    for op in ops:
        t, U = op_matrix(op, d, params)
        apply(out, d, n, t, U)
    return out


def number_weights_diag(d, n: int, weights) -> np.ndarray:
    """Diagonal of O = sum_q w_q N_q: entry i is sum_q w_q i_q."""
    dims = dims_of(d, n)
    N = int(np.prod(dims, dtype=np.int64))
    i = np.arange(N, dtype=np.int64)
    diag = np.zeros(N)
    S = 1
    for q in range(n - 1, -1, -1):
        diag += float(weights[q]) * ((i // S) % dims[q])
        S *= dims[q]
    return diag


def loss(psi, d, n, weights) -> float:
    """sum_q w_q <N_q>."""
    e = expect_number(psi, d, n)
    return float(np.dot(np.asarray(weights, dtype=float), e))


def grad_bruteforce(ops, d, n: int, params, weights, psi0=None, slots=None) -> np.ndarray:
    """dL/dtheta_p for L = sum_q w_q <N_q>, by explicit derivative circuits."""
    params = np.asarray(params, dtype=float)
    P = len(params)
    slots = list(range(P) if slots is None else slots)
    start = basis(d, n, 0) if psi0 is None else np.array(psi0, dtype=np.complex128)
    uses = {}
    for l, op in enumerate(ops):
        if op.kind in ("rot", "crot") and op.param >= 0:
            uses.setdefault(op.param, []).append(l)
    # prefix[l] = state before gate l, kept only for the gates of the
    # requested slots (the full list would hold one state per gate)
    need = {l for p in slots for l in uses.get(p, [])}
    prefix = {}
    cur = start.copy()
    for l, op in enumerate(ops):
        if l in need:
            prefix[l] = cur.copy()
        t, U = op_matrix(op, d, params)
        apply(cur, d, n, t, U)
    final = cur
    Odiag = number_weights_diag(d, n, weights)
    O_psi = Odiag * final
    g = np.zeros(len(slots))
    for out_i, p in enumerate(slots):
        dpsi = np.zeros_like(final)
        for l in uses.get(p, []):
            v = prefix[l].copy()
            t, dU = op_matrix(ops[l], d, params, deriv=True)
            apply(v, d, n, t, dU)
            for op in ops[l + 1:]:
                t2, U2 = op_matrix(op, d, params)
                apply(v, d, n, t2, U2)
            dpsi += v
        g[out_i] = 2.0 * inner(O_psi, dpsi).real
    return g


def grad_fd(ops, d, n: int, params, weights, h: float = 1e-5, psi0=None, slots=None) -> np.ndarray:
    """Central finite differences (L(theta + h e_p) - L(theta - h e_p)) / 2h."""
    params = np.asarray(params, dtype=float)
    slots = range(len(params)) if slots is None else slots
    out = []
    for p in slots:
        tp = params.copy(); tp[p] += h
        tm = params.copy(); tm[p] -= h
        lp = loss(run(ops, d, n, psi0, tp), d, n, weights)
        lm = loss(run(ops, d, n, psi0, tm), d, n, weights)
        out.append((lp - lm) / (2.0 * h))
    return np.array(out)


def sample(probs, uniforms) -> np.ndarray:
    """Histogram of samples from a discrete distribution by its inverse
    CDF: sample s falls in the first bin whose cumulative probability exceeds
    uniforms[s] times the total."""
    probs = np.asarray(probs, dtype=float)
    cdf = np.cumsum(probs)
    x = np.asarray(uniforms, dtype=float) * cdf[-1]
    idx = np.searchsorted(cdf, x, side="right")
    return np.bincount(np.minimum(idx, len(probs) - 1), minlength=len(probs)).astype(np.int64)
