"""GB300-native state-vector simulator for driven spin chains (arXiv 2111.08044)."""
