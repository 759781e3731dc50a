"""GB300-native image-plane single-pulse search (DSA-110 NSFRB, arXiv 2510.18136)."""
