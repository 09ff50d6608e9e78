"""Plain FP64 reference of the relativistic SHASTA step (test infrastructure only)."""
