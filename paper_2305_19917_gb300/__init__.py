"""GB300-native triangular solver (TRSM) with recursive, iterative and
blocked decompositions (arXiv 2305.19917, Sections IV-V).

Importing the package loads nothing; ``paper_2305_19917_gb300.api`` loads the
CUDA library (and fails loudly if it is missing).
"""
