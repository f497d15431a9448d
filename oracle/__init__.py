"""FP64 CPU oracle for the batched chemical source term (test infrastructure only)."""
