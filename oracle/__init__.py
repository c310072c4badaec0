"""FP64 CPU oracle (test infrastructure only; see laker_oracle)."""
