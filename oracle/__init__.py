"""FP64 CPU oracle (test infrastructure only; see egn_oracle.c)."""
