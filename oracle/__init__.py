"""FP64 CPU oracle of the PB hot path -- test infrastructure only (see oracle.py)."""
