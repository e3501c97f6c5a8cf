"""Seeded synthetic circuits: the inputs shared by the oracle and the GPU path.

This module draws random numbers and lays out gate lists; it holds none of the
simulator's arithmetic (no gate matrix is built here, except that a
Haar-random unitary *is* the drawn input of a custom gate).  Both the CPU
oracle and the CUDA library consume the same ``Op`` lists, so both sides see
identical angles and matrices.

Gate kinds (paper, Appendix B):
  'h'    Fourier gate on qudit q
  'x'    generalised NOT X_s (shift s = ``power``)
  'z'    phase-shift / clock P^p (power p = ``power``)
  'rot'  rotation exp(-i theta S/2) on levels (j, k); axis 'x', 'y', 'z'
         (two-level diagonal) or 'g' (Gell-Mann diagonal S_z^j, k unused)
  'crot' controlled rotation sum_m |m><m| (x) R(m theta) on (control, target)
  'sum'  generalised CNOT |c>|t> -> |c>|t + c mod d>
  'swap' generalised SWAP
  'u'    custom d^k x d^k matrix on the listed qudits (first = most significant)
  'mcx'  multi-controlled X^s on qudits (c_1, .., c_k, t): t += s * c_1 ... c_k
  'mcu'  d_t x d_t ``matrix`` on the last qudit when control i is at ``levels[i]``

A rotation either carries a fixed angle ``theta`` or names a slot ``param`` of
a parameter vector supplied at run time.

Workload recipes (seeded; one master seed, each workload xors in its id):
  * ``layered_circuit``   -- d=3, n=6, 20 layers of Fourier / RX RY RZ on
    level pairs (0,1), (1,2) / nearest-neighbour SUM chain, angles U[0, 2pi).
  * ``random_circuit``    -- 200 gates drawn uniformly from {Haar U, level-pair
    rotation, clock Z, shift X, SUM-or-controlled-RY}, qudits uniform.
  * ``variational_ansatz``-- L layers of RY, RZ on (0,1), (1,2) on every qudit
    then a SUM ring or chain; parameter slots numbered layer, kind, qudit.
  * ``batch_circuits``    -- many small circuits of uneven d, n, L with
    per-sample encoding angles and a shared trainable-angle table.
  * ``vqa_circuit`` / ``vqa_batch`` -- the paper's VQA circuit (Fourier,
    RZ encoding, rotation block R1/R2/R3, CNOT fan-out from qudit 0, rotation
    block) for a batch of samples with uniform stand-in encoding angles.
  * ``mixed_random_circuit`` / ``mixed_ansatz`` -- circuits on registers that
    mix qudit dimensions (dims[q] per qudit).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

MASTER_SEED = 20240917
TWO_PI = 2.0 * math.pi


@dataclass(frozen=True)
class Op:
    kind: str
    qudits: Tuple[int, ...]
    j: int = 0
    k: int = 1
    axis: str = ""
    theta: float = 0.0
    param: int = -1
    power: int = 1
    matrix: Optional[np.ndarray] = field(default=None, compare=False, repr=False)
    levels: Tuple[int, ...] = ()

    def angle(self, params: Optional[Sequence[float]] = None) -> float:
        if self.param >= 0:
            if params is None:
                raise ValueError("op uses parameter slot %d but no parameters given" % self.param)
            return float(params[self.param])
        return float(self.theta)


def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random d x d unitary (Mezzadri 2007): QR of a complex Ginibre matrix
    with N(0, 1/2) components, columns rephased by r_ii / |r_ii|."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)


def _pair(d: int, rng: np.random.Generator) -> Tuple[int, int]:
    a, b = rng.choice(d, size=2, replace=False)
    return (int(min(a, b)), int(max(a, b)))


def layered_circuit(d: int = 3, n: int = 6, layers: int = 20, seed: int = MASTER_SEED ^ 1) -> List[Op]:
    """Fourier on all qudits; RX, RY, RZ on level pairs (0,1), (1,2) on all
    qudits (angles U[0, 2pi), drawn layer -> kind -> qudit); SUM(q, q+1) chain."""
    rng = np.random.default_rng(seed)
    ops: List[Op] = []
    pairs = [(0, 1), (1, 2)] if d > 2 else [(0, 1)]
    for _ in range(layers):
        for q in range(n):
            ops.append(Op("h", (q,)))
        for axis in ("x", "y", "z"):
            for (j, k) in pairs:
                for q in range(n):
                    ops.append(Op("rot", (q,), j=j, k=k, axis=axis, theta=float(rng.uniform(0.0, TWO_PI))))
        for q in range(n - 1):
            ops.append(Op("sum", (q, q + 1)))
    return ops


RANDOM_KINDS = ("u", "rot", "z", "x", "sum_or_cry")


def random_gate(kind: str, d: int, n: int, rng: np.random.Generator, target: Optional[int] = None) -> Op:
    """One gate of the random-sequence workload.  ``target`` pins the (target)
    qudit for the per-target sweep; otherwise it is uniform."""
    q = int(rng.integers(n)) if target is None else int(target)
    if kind == "u":
        return Op("u", (q,), matrix=haar_unitary(d, rng))
    if kind == "rot":
        axis = ("x", "y", "z")[int(rng.integers(3))]
        j, k = _pair(d, rng)
        return Op("rot", (q,), j=j, k=k, axis=axis, theta=float(rng.uniform(0.0, TWO_PI)))
    if kind == "z":
        return Op("z", (q,), power=int(rng.integers(1, d)))
    if kind == "x":
        return Op("x", (q,), power=int(rng.integers(1, d)))
    if kind in ("sum_or_cry", "sum", "cry"):
        c = int(rng.integers(n - 1))
        if c >= q:
            c += 1
        pick_sum = (rng.random() < 0.5) if kind == "sum_or_cry" else (kind == "sum")
        if pick_sum:
            return Op("sum", (c, q))
        j, k = _pair(d, rng)
        return Op("crot", (c, q), j=j, k=k, axis="y", theta=float(rng.uniform(0.0, TWO_PI)))
    raise ValueError(kind)


def random_circuit(d: int, n: int, n_gates: int = 200, seed: int = MASTER_SEED ^ 2) -> List[Op]:
    """Random sequence: each gate's kind uniform over RANDOM_KINDS, then its
    qudits, levels and angle; the seed also folds in (d, n)."""
    rng = np.random.default_rng([seed, d, n])
    return [random_gate(RANDOM_KINDS[int(rng.integers(len(RANDOM_KINDS)))], d, n, rng) for _ in range(n_gates)]


def variational_ansatz(d: int, n: int, layers: int, entangler: str = "ring",
                       first_param: int = 0) -> Tuple[List[Op], int]:
    """Per layer: RY(0,1), RY(1,2), RZ(0,1), RZ(1,2) on every qudit (pairs with
    level 2 are skipped when d = 2), then SUM(q, q+1) for q = 0..n-2 and, for a
    ring, SUM(n-1, 0).  Parameter slot = first_param + running index in the
    order layer -> rotation kind -> qudit.  Returns (ops, parameter count)."""
    kinds = [("y", 0, 1), ("y", 1, 2), ("z", 0, 1), ("z", 1, 2)]
    if d == 2:
        kinds = [kk for kk in kinds if kk[2] < 2]
    ops: List[Op] = []
    p = first_param
    for _ in range(layers):
        for (axis, j, k) in kinds:
            for q in range(n):
                ops.append(Op("rot", (q,), j=j, k=k, axis=axis, param=p))
                p += 1
        for q in range(n - 1):
            ops.append(Op("sum", (q, q + 1)))
        if entangler == "ring" and n > 2:
            ops.append(Op("sum", (n - 1, 0)))
    return ops, p - first_param


def normal_angles(count: int, sigma: float = 1.0, seed: int = MASTER_SEED ^ 3) -> np.ndarray:
    rng = np.random.default_rng([seed, count])
    return sigma * rng.standard_normal(count)


@dataclass
class BatchCircuit:
    d: int
    n: int
    layers: int
    ops: List[Op]           # encoding + ansatz; params index the global vector
    n_params: int


def batch_circuits(count: int = 4096, seed: int = MASTER_SEED ^ 4,
                   d_range=(2, 5), n_range=(4, 10), l_range=(2, 6),
                   max_layers: int = 6, max_n: int = 10):
    """Uneven batch.  Per sample: d ~ U{2..5}, n ~ U{4..10}, L ~ U{2..6}.
    Circuit = Fourier on every qudit, then RZ^{01}(x_q) with a per-sample
    encoding angle x_q ~ U[0, pi), then the variational ansatz (SUM ring) whose
    angles come from one shared table theta[L][kind][q] ~ N(0, 0.1) (each sample
    uses its prefix).  Parameter vector layout: [shared table (max_layers * 4 *
    max_n)] + [encoding angles of every sample, max_n per sample].
    Returns (circuits, params)."""
    rng = np.random.default_rng(seed)
    n_shared = max_layers * 4 * max_n
    shared = 0.1 * rng.standard_normal(n_shared)
    circuits: List[BatchCircuit] = []
    enc = np.zeros((count, max_n))
    for s in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        L = int(rng.integers(l_range[0], l_range[1] + 1))
        enc[s, :n] = rng.uniform(0.0, math.pi, size=n)
        ops: List[Op] = [Op("h", (q,)) for q in range(n)]
        for q in range(n):
            ops.append(Op("rot", (q,), j=0, k=1, axis="z", param=n_shared + s * max_n + q))
        kinds = [("y", 0, 1), ("y", 1, 2), ("z", 0, 1), ("z", 1, 2)]
        for layer in range(L):
            for kind, (axis, j, k) in enumerate(kinds):
                if d == 2 and k >= 2:
                    continue
                for q in range(n):
                    slot = (layer * 4 + kind) * max_n + q
                    ops.append(Op("rot", (q,), j=j, k=k, axis=axis, param=slot))
            for q in range(n - 1):
                ops.append(Op("sum", (q, q + 1)))
            if n > 2:
                ops.append(Op("sum", (n - 1, 0)))
        circuits.append(BatchCircuit(d, n, L, ops, 0))
    params = np.concatenate([shared, enc.reshape(-1)])
    return circuits, params


def uniform_state(d, n: int, seed: int = MASTER_SEED ^ 5) -> np.ndarray:
    """Random normalised complex128 state of d^n amplitudes (Gaussian
    entries); d may be a sequence of per-qudit dimensions."""
    if isinstance(d, (int, np.integer)):
        rng = np.random.default_rng([seed, d, n])
        N = d ** n
    else:
        rng = np.random.default_rng([seed] + [int(x) for x in d])
        N = int(np.prod([int(x) for x in d], dtype=np.int64))
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return (v / np.linalg.norm(v)).astype(np.complex128)


def rotation_block(d: int, n: int, variant: str, first_param: int) -> Tuple[List[Op], int]:
    """One rotation block of the VQA circuit ("Variational quantum algorithm"
    section), on every qudit, RX first, then RY, then RZ:
      R1: level pair (0,1) for x, y and the level-pair z;
      R2: x and y on pairs (0,k), k = 1..d-1; z as Gell-Mann S_z^j, j = 1..d-1;
      R3: x and y on every pair (j,k); z as Gell-Mann S_z^j, j = 1..d-1.
    Returns (ops, parameters used); slots are numbered from first_param in op order."""
    if variant == "R1":
        xy = [(0, 1)]
    elif variant == "R2":
        xy = [(0, k) for k in range(1, d)]
    elif variant == "R3":
        xy = [(j, k) for j in range(d) for k in range(j + 1, d)]
    else:
        raise ValueError(variant)
    ops: List[Op] = []
    p = first_param
    for axis in ("x", "y"):
        for (j, k) in xy:
            for q in range(n):
                ops.append(Op("rot", (q,), j=j, k=k, axis=axis, param=p))
                p += 1
    if variant == "R1":
        for q in range(n):
            ops.append(Op("rot", (q,), j=0, k=1, axis="z", param=p))
            p += 1
    else:
        for j in range(1, d):
            for q in range(n):
                ops.append(Op("rot", (q,), j=j, axis="g", param=p))
                p += 1
    return ops, p - first_param


def vqa_circuit(d: int, n: int, variant: str, enc_first: int, theta_first: int) -> Tuple[List[Op], int]:
    """The VQA circuit of the paper's figure: Fourier on every qudit, RZ^{01}
    data encoding (slots enc_first + q), a rotation block, CNOT (SUM) from
    qudit 0 to every other qudit, a second rotation block.  Returns (ops,
    trainable parameters used from theta_first)."""
    ops: List[Op] = [Op("h", (q,)) for q in range(n)]
    ops += [Op("rot", (q,), j=0, k=1, axis="z", param=enc_first + q) for q in range(n)]
    b1, p1 = rotation_block(d, n, variant, theta_first)
    ops += b1
    ops += [Op("sum", (0, q)) for q in range(1, n)]
    b2, p2 = rotation_block(d, n, variant, theta_first + p1)
    ops += b2
    return ops, p1 + p2


def vqa_batch(count: int, d: int, n: int, variant: str, seed: int = MASTER_SEED ^ 6):
    """`count` samples of one VQA circuit shape: per-sample encoding angles
    U[0, pi) (stand-ins for the Iris / MNIST features the paper encodes) and
    shared trainable angles N(0, 0.1).  Parameter vector = [trainable | n
    encodings per sample].  Returns (circuits, params)."""
    rng = np.random.default_rng([seed, d, n, ord(variant[-1])])
    _, P = vqa_circuit(d, n, variant, 0, 0)
    theta = 0.1 * rng.standard_normal(P)
    enc = rng.uniform(0.0, math.pi, size=(count, n))
    template, _ = vqa_circuit(d, n, variant, 0, 0)   # ops are frozen: shared between samples
    circuits = []
    for s in range(count):
        ops = list(template)
        ops[n:2 * n] = [Op("rot", (q,), j=0, k=1, axis="z", param=P + s * n + q) for q in range(n)]
        circuits.append(BatchCircuit(d, n, 2, ops, P))
    return circuits, np.concatenate([theta, enc.reshape(-1)])


MIXED_KINDS = ("u", "rot", "z", "x", "h", "sum", "crot", "swap", "u2")


def mixed_random_gate(kind: str, dims: Sequence[int], rng: np.random.Generator,
                      target: Optional[int] = None) -> Op:
    """One gate on a register whose qudit q has dimension dims[q]: levels and
    powers are drawn within the target's dimension; a SWAP needs two qudits of
    equal dimension (a SUM is drawn when the target has no such partner); a
    two-qudit Haar U needs d_a * d_b <= 64."""
    n = len(dims)
    q = int(rng.integers(n)) if target is None else int(target)
    d = int(dims[q])
    if kind == "u":
        return Op("u", (q,), matrix=haar_unitary(d, rng))
    if kind == "rot":
        axis = ("x", "y", "z", "g")[int(rng.integers(4))]
        if axis == "g":
            return Op("rot", (q,), j=int(rng.integers(1, d)), axis="g", theta=float(rng.uniform(0.0, TWO_PI)))
        j, k = _pair(d, rng)
        return Op("rot", (q,), j=j, k=k, axis=axis, theta=float(rng.uniform(0.0, TWO_PI)))
    if kind == "z":
        return Op("z", (q,), power=int(rng.integers(1, d)))
    if kind == "x":
        return Op("x", (q,), power=int(rng.integers(1, d)))
    if kind == "h":
        return Op("h", (q,))
    c = int(rng.integers(n - 1))
    if c >= q:
        c += 1
    if kind == "swap":
        same = [p for p in range(n) if p != q and dims[p] == d]
        if not same:
            return Op("sum", (c, q))
        return Op("swap", (int(same[int(rng.integers(len(same)))]), q))
    if kind == "sum":
        return Op("sum", (c, q))
    if kind == "crot":
        axis = ("x", "y", "z", "g")[int(rng.integers(4))]
        if axis == "g":
            return Op("crot", (c, q), j=int(rng.integers(1, d)), axis="g", theta=float(rng.uniform(0.0, TWO_PI)))
        j, k = _pair(d, rng)
        return Op("crot", (c, q), j=j, k=k, axis=axis, theta=float(rng.uniform(0.0, TWO_PI)))
    if kind == "u2":
        if dims[c] * d > 64:
            return Op("sum", (c, q))
        return Op("u", (c, q), matrix=haar_unitary(int(dims[c]) * d, rng))
    raise ValueError(kind)


def mixed_random_circuit(dims: Sequence[int], n_gates: int = 200, seed: int = MASTER_SEED ^ 7,
                         kinds: Sequence[str] = MIXED_KINDS) -> List[Op]:
    """Random sequence on a mixed-dimension register (section "Code style":
    Circuit(dim=[2,3,4])): kind uniform over `kinds`, then qudits, levels,
    angle; the seed folds in the dimensions."""
    rng = np.random.default_rng([seed] + [int(x) for x in dims])
    return [mixed_random_gate(kinds[int(rng.integers(len(kinds)))], dims, rng) for _ in range(n_gates)]


def mixed_ansatz(dims: Sequence[int], layers: int, first_param: int = 0) -> Tuple[List[Op], int]:
    """Variational layers on a mixed register: Fourier on every qudit (first
    layer only); per layer RX(0,1), RY(0,1) and Gell-Mann RZ^(d_q - 1) on every
    qudit, then controlled RY(0,1) from q to q+1 and SUM(q+1, q) for
    q = 0..n-2.  Parameter slots run layer -> kind -> qudit.  Returns (ops,
    parameter count)."""
    n = len(dims)
    ops: List[Op] = [Op("h", (q,)) for q in range(n)]
    p = first_param
    for _ in range(layers):
        for axis in ("x", "y"):
            for q in range(n):
                ops.append(Op("rot", (q,), j=0, k=1, axis=axis, param=p))
                p += 1
        for q in range(n):
            ops.append(Op("rot", (q,), j=int(dims[q]) - 1, axis="g", param=p))
            p += 1
        for q in range(n - 1):
            ops.append(Op("crot", (q, q + 1), j=0, k=1, axis="y", param=p))
            p += 1
            ops.append(Op("sum", (q + 1, q)))
    return ops, p - first_param
