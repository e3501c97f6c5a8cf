"""CPU oracle for the qudit state-vector path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library:
the C file ``qf_oracle.c`` builds every gate from the paper's Appendix B
definitions and applies it with explicit loops in complex128.

Parity pins (see tests/test_oracle_*.py): Kronecker-product brute force on tiny
registers, the matrices the paper prints (D=2 rotations, D=3 and D=4 RX^{1,2},
Fourier, phase), textbook qubit gates at d=2, matrix exponentials of the
Gell-Mann generators, invariants (unitarity, X^d = I, ZX = wXZ, H^4 = I, SUM^d =
I, GHZ), and the closed-form Deutsch-Jozsa and Grover outcomes.
"""
from . import sim  # noqa: F401
