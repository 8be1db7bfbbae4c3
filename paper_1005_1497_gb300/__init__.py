"""GB300-native exact digital circular convolution (Chandra, arXiv 1005.1497)."""
