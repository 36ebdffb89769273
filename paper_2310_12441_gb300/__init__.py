"""BootMMPM on GB300: blind rotation of a polynomial-vector test vector by
RGSW-encrypted monic monomial permutation matrices, sample extraction and
LWE key switching (arXiv 2310.12441, Algorithm 1), as hand-written sm_103a
CUDA behind a C ABI (libbootmmpm.so, include/bootmmpm.h).

Importing the package loads nothing; `paper_2310_12441_gb300.api` loads the
CUDA library and fails loudly when it is missing.
"""
from . import params, synth  # noqa: F401
