"""GB300-native 3D Gaussian Splatting training hot path (BalanceGS, arXiv 2510.14564)."""
