"""GB300-native Link-wise Artificial Compressibility Method (LW-ACM).

The compute path is the C-ABI library ``liblwacm.so`` built from ``csrc/``
(hand-written sm_103a CUDA kernels); ``lwacm.py`` is a thin ctypes binding with
the same call names. Nothing here falls back to a CPU implementation: every
entry point raises if the CUDA library is missing. Importing the package does
not load the library; ``paper_1111_2142_gb300.lwacm`` does, on first use.
"""
