"""FP64 CPU oracle of the IBM step.  Test infrastructure only (see oracle.py)."""
