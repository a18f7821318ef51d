"""Seeded synthetic inputs shared by the oracle tests and the device tests.

Nothing here computes any part of the community integration method.
"""
from .graphs import (Graph, complete_graph_communities, equal_sizes, hash_sbm_graph, hierarchical_sbm_graph,
                     lognormal_sizes,
                     random_labels_graph, rng_for, sbm_graph)
from .workloads import (CuckerSmaleWorkload, EnsembleWorkload, KuramotoWorkload, as_fp32_values,
                        cached, cucker_smale, ensemble_instance, ensemble_instance_shape,
                        kuramoto_ensemble, kuramoto_ho, kuramoto_lognormal, kuramoto_sbm_small)

__all__ = [
    "Graph", "complete_graph_communities", "equal_sizes", "hash_sbm_graph", "hierarchical_sbm_graph",
    "lognormal_sizes",
    "random_labels_graph", "rng_for", "sbm_graph", "CuckerSmaleWorkload",
    "KuramotoWorkload", "as_fp32_values", "cached", "cucker_smale", "kuramoto_ho",
    "kuramoto_lognormal", "kuramoto_sbm_small", "EnsembleWorkload", "kuramoto_ensemble",
    "ensemble_instance", "ensemble_instance_shape",
]
