"""GB300-native SCD + LP-rounding solver (arXiv 1311.2661)."""
