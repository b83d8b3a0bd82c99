"""FP64 brute-force CPU oracle -- test infrastructure only (see oracle.py)."""
