"""GB300-native hot path of the LB freezing method of arXiv 2510.18688."""
