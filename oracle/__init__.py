"""CPU oracle (test infrastructure only; see hss_oracle's header)."""
