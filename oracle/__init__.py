"""FP64 CPU oracle of the implicit r-z PIC/MCC step (test infrastructure only)."""
