"""CPU oracle for the sigma cuts (test infrastructure only; see oracle.py)."""
