"""GB300-native diag(H^-1) solver for the IDMFT Dyson equation (low-rank correction method)."""
