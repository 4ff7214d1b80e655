"""FP64 CPU oracle of the coupled D3Q19 LBM step (test infrastructure only)."""
