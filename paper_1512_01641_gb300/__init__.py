"""GB300-native comparable-corpus miner (Wolk & Marasek, arXiv:1512.01641).

Hot path: dictionary-overlap sentence similarity (Section 4) and
Needleman-Wunsch sentence alignment with an acceptance threshold
(Section 5.1), as hand-written sm_103a CUDA kernels behind the C ABI in
include/miner.h.  ``miner`` is the Python binding; ``synth`` draws seeded
synthetic corpora.  Importing the package loads nothing; the library is
loaded on first use.
"""
__all__ = ["miner", "synth", "build"]
