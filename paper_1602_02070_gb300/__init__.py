"""GB300 (sm_103a) compressive PCA on graphs (arXiv 1602.02070).

The computation lives in libcpca.so (C ABI: include/cpca.h); this package is
its thin binding plus the end-to-end composition of Table "tab:cpca".
"""
from .capi import (CPCA_ERR_CAPACITY, CPCA_ERR_CUDA, CPCA_ERR_INVALID_ARG, CPCA_ERR_NONFINITE,  # noqa: F401
                   CPCA_ERR_NOT_CONVERGED, CPCA_ERR_SINGULAR, CPCA_ERR_TIMEOUT,
                   CPCA_ERR_WORKSPACE, CPCA_OK, LAP_COMBINATORIAL, LAP_NORMALIZED, Batch, CpcaError, Csr,
                   alt_params, cpca_alternate_decode, cpca_cluster_decode, cpca_decode, cpca_subspace_project, cpca_decode_backward, cpca_frpcag_backward, cpca_frpcag_solve, cpca_frpcag_solve_noalloc, cpca_frpcag_status,
                   debug_set_barrier_spin_limit,
                   cpca_knn_graph, cpca_kron_reduce, cpca_sample, decode_params,
                   exported_names, frpcag_params, knn_last_bruteforce, knn_last_err_rel, knn_last_uncertified, launch_count, lib,
                   profile_enable,
                   profile_read)
from .pipeline import cpca_pipeline, rho_of  # noqa: F401
