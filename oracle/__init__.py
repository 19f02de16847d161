"""CPU FP64 oracle (test infrastructure only; see emfuse_oracle.py)."""
