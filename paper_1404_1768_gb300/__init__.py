"""GB300-native oblique-projection FEAST (placeholder; binding added below)."""
