"""GB300-native engine for the quantum-trajectory hot path of QTraj 1.0 (arXiv:2107.06147).

The compute path is the C-ABI library ``libqtraj.so`` (hand-written sm_103a CUDA); ``qtraj.py`` is
its thin ctypes binding.  Import ``paper_2107_06147_gb300.qtraj`` for the engine; ``inputs`` holds
the seeded synthetic workloads.
"""
