"""FP64 CPU oracle of the method (test infrastructure only; see oracle.py)."""
