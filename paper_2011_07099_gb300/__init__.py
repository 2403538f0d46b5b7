"""GB300-native natively periodic FMM (Gnedin, arXiv:2011.07099)."""
