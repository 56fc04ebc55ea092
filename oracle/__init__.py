"""FP64 CPU oracle for EDAA (test infrastructure only; never imported by the
library or its Python binding)."""
