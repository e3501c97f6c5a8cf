"""GB300-native qudit state-vector engine (QuForge hot path, arXiv 2409.17716)."""
