"""GB300-native forcing-based free-energy D2Q9 lattice Boltzmann step."""
