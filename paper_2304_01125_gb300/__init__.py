"""GB300-native FFT crystal-plasticity phase-field fatigue solver."""
