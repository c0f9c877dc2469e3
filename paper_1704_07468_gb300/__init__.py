"""GB300-native gapped k-mer string kernel (GaKCo, arXiv 1704.07468)."""
