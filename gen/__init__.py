"""Seeded synthetic workloads for the pDCA graph Ginzburg-Landau solver.

This package builds the *inputs* of the method: feature data (points or image
patches), the k-nearest-neighbour graph with Gaussian weights (Sec. 2.2 of the
paper, eq. for K(i,j) and the proximity indicators N_s / N_c), the labelled set
and the ground truth.  It contains none of the solver's arithmetic (no
Laplacian, no DCA step, no preconditioner); the oracle and the CUDA library
both consume the same CSR arrays produced here.
"""

from .workloads import (  # noqa: F401
    Workload,
    WORKLOADS,
    make_workload,
    two_moons,
    ellipse_image,
    voronoi_image,
    gmm_points,
    knn_graph_points,
    knn_graph_image,
    sample_labels,
    random_graph,
    banded_graph,
    csr_from_pairs,
)
