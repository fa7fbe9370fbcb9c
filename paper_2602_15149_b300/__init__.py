"""B300-native total-Lagrangian SPH solid step (arXiv 2602.15149).

The compute path is the C-ABI library ``libtlsph.so`` built from ``csrc/``
(sm_103a CUDA); :mod:`paper_2602_15149_b300.tlsph` is its thin ctypes binding
and :mod:`paper_2602_15149_b300.workloads` builds seeded synthetic inputs.
Import the submodules directly: the package itself loads nothing.
"""
