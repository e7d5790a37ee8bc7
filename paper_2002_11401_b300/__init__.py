"""flatspin relax loop on B300: geometry, neighbour tensors, field-and-margin
sweep and greedy single-flip relaxation as hand-written CUDA behind a C ABI.

Importing the package loads nothing; ``paper_2002_11401_b300.binding`` loads the
compiled library (and fails loudly if it is missing).
"""
__all__ = ["binding", "inputs"]
