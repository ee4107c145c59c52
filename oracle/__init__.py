"""FP64 CPU oracle (test infrastructure only; see dwf_oracle.py)."""
