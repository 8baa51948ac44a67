"""GB300-native Stokeslet + stresslet treecode (arXiv:1811.12498)."""
