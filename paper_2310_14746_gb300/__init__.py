"""GB300-native homogenized lattice BGK (HBGK) stream-collide library."""
