"""CPU oracle for the pointerless level-wise wavelet tree (test infrastructure only)."""
