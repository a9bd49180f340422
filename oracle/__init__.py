"""CPU oracle for the data-parallel GKR prover (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library; see ``sisu_oracle.c`` (the plain C oracle) and ``brute.py`` (a
pure-Python brute-force prover that pins it on micro circuits).
"""
from .binding import Oracle, build_oracle, LIB_PATH  # noqa: F401
