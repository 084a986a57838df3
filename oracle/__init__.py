"""FP64 CPU oracle for RQRCP -- test infrastructure only (see oracle.py)."""
