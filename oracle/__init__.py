"""FP64 CPU oracle -- test infrastructure only (see fdtd_oracle.c)."""
