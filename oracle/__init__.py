"""FP64 CPU oracle of the TLSPH solid step (arXiv 2602.15149).

TEST INFRASTRUCTURE ONLY.  This package is the parity reference for the CUDA
library and the timed CPU baseline; only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import it.  It shares no code with the CUDA path
(``paper_2602_15149_b300``): the two only meet in the seeded input
generators of ``paper_2602_15149_b300.workloads``, which hold none of the
method's arithmetic.

Parity status of the oracle's functions (what pins each one is in
``tests/test_oracle_pins.py``): every function is pinned by a closed form,
an invariant or a brute-force check, except the pre-existing notch cut,
whose geometric reading (bond removal) is pinned only by exact
segment-intersection cases, not by a physical result ("parity unpinned"
for its physical effect).
"""
from .oracle import Oracle, OracleMaterial, build_oracle, load_oracle  # noqa: F401
