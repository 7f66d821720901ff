"""GB300-native TMFG construction and APSP over the TMFG (arXiv 2408.09399)."""
