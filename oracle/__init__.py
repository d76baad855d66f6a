"""CPU FP64 oracle for the low-sync block Arnoldi solver (test infrastructure only)."""
