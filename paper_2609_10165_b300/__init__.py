"""B300-native direct ghost-cell reconstruction for Cartesian embedded boundaries."""
