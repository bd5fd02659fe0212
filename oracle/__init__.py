"""FP64 CPU oracle (test infrastructure only; see ftcg_oracle)."""
