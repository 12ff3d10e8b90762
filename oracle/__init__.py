"""FP64 CPU oracle for GRTX Gaussian ray tracing (test infrastructure only; see oracle.py)."""
