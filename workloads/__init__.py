"""Seeded synthetic workloads (sorted distinct uint32 lists, query term sets,
arrival times) shaped like the paper's experiments.  Holds no coding or
intersection arithmetic; both the oracle and the CUDA path consume it."""
from .workloads import (  # noqa: F401
    build_workloads, uniform, clustered, many, pair_short, zipf_lengths,
    queries, poisson_arrivals, stepped_walk, CLUEWEB_TERM_WEIGHTS_2_5,
    CLUEWEB_TERM_WEIGHTS_2_8,
)
