"""Seeded synthetic CGGM problems (inputs only).

This module draws X, Y and the true (Lambda, Theta) of the workloads the solver is
measured on, by sampling the conditional Gaussian model of Section 2.1 in the form
y | x ~ N(-Lambda^-1 Theta^T x, Lambda^-1) (the form the negative log-likelihood of
Eq. 1 belongs to).  It holds none of the solver's arithmetic: no objective,
gradient, active set, coordinate step or line search lives here.  The CPU oracle
tests and the CUDA path take their inputs from here and from nowhere else.
"""
from .problems import (  # noqa: F401
    Problem,
    chain_precision,
    random_sparse_precision,
    sparse_theta,
    gaussian_X,
    genotype_X,
    sample_Y,
    make_problem,
    workload,
    WORKLOADS,
    serving_requests,
    clustered_precision,
    clustered_theta,
    clustered_problem,
)
