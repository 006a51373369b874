"""CPU FP64 oracle (test infrastructure only; see bn_oracle.c)."""
