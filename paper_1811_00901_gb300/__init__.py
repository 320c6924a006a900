"""GB300-native spin-image generation with dynamic loop scheduling."""
