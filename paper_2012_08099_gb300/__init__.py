"""GB300-native Discrete Projection Moment library (placeholder, filled in below)."""
