"""GB300-native randomized QR with column pivoting (RQRCP).

The compute path is the C-ABI library ``librqrcp.so`` built from ``csrc/`` (CUDA for
sm_103a); ``binding`` marshals arguments to it.  Importing this package loads nothing:
the library is loaded on first use and a missing library raises an error.
"""
__all__ = ["binding", "inputs"]
