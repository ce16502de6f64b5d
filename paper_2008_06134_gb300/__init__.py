"""GB300-native slice-based illuminated ray casting (arXiv 2008.06134)."""
