"""GB300-native differentiable Voronoi ray tracing (placeholder, filled below)."""
