"""FP64 CPU oracle (test infrastructure only; see qaoa_oracle.py)."""
