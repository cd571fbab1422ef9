"""Seeded synthetic Markov chains (inputs only; no step of the solver lives here).

Both the CPU oracle and the CUDA path read their inputs from this package, so it
holds nothing but the test problems of Section 5.1 of the paper and the batched
mixtures built from them.  Every generator returns a column-stochastic transition
matrix A in CSR form whose row i lists the source states j with a_ij = P(j -> i).
"""

from .chains import (  # noqa: F401
    Chain,
    grid_walk,
    tandem_queue,
    birth_death,
    delaunay_walk,
    random_birth_death,
    batched_mixture,
    tandem_training_set,
)
