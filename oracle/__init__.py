"""FP64 CPU oracle (test infrastructure only; see hhl_oracle's module docstring)."""
