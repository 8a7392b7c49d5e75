"""GB300-native locally relaxed entropy-stable RK step (placeholder, filled below)."""
