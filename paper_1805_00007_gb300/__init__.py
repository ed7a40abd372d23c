"""GB300-native D2Q9 lattice Boltzmann solver for the Cahn-Hilliard equation (Zhang, Guo & Liang)."""
