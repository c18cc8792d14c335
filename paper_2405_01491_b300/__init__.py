"""ANI-2x-style energy and forces (FeNNol, arXiv 2405.01491) as hand-written sm_103a CUDA.

Importing the package loads nothing native; ``paper_2405_01491_b300.fnn``
loads the C-ABI library and fails loudly when it is missing.
"""
