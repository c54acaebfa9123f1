"""GB300-native geometric multigrid for the finite-difference Poisson equation."""
