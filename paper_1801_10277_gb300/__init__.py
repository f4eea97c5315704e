"""GB300-native Celeste ELBO / gradient / Hessian / trust-region Newton hot path.

Importing the package loads nothing native; ``paper_1801_10277_gb300.celeste`` binds
the CUDA library (built by ``__graft_entry__.build()``) and fails loudly when it is
missing.
"""
