"""GB300-native moment-encoded multi-level lattice Boltzmann hot path."""
