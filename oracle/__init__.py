"""Independent CPU oracle of the RSR hot path (test infrastructure only; see oracle.py)."""
