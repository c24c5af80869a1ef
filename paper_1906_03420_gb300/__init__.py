"""GB300-native (sm_103a) subgraph isomorphism search: signature filtering and
vertex-oriented joins (Sun et al., arXiv 1906.03420), behind a C ABI
(include/gsi.h).  This package is the thin Python binding; the work runs in
libgsi.so's CUDA kernels."""
from .gsi import (GSI_EBUSY, GSI_ECANCELLED, GSI_ECAPPED, GSI_ECUDA, GSI_EINVAL, GSI_ENOMEM, GSI_ETIMEOUT, GSI_OK,
                  GSI_HOMOMORPHISM, GSI_ISOMORPHISM, GSI_EDGE_HOST_ONLY, GSI_ISECT_BSEARCH, GSI_ISECT_MERGE,
                  GSI_ISECT_BITMAP,
                  EXPORTED, EdgeGraph, Graph, batch_autotune, batch_autotune_full, GsiError, PreparedBatch, QueryArrays, Result, Server, c_stats, last_error, lib_path, load,
                  plan_order, query_signatures, selftest_wait_timeout, version)

__all__ = ["EdgeGraph", "Graph", "batch_autotune", "batch_autotune_full", "GsiError", "PreparedBatch", "QueryArrays", "Result", "Server", "c_stats", "load", "lib_path", "plan_order",
           "query_signatures", "selftest_wait_timeout", "version", "last_error", "EXPORTED", "GSI_OK", "GSI_EINVAL", "GSI_ENOMEM",
           "GSI_ECAPPED", "GSI_ETIMEOUT", "GSI_ECANCELLED", "GSI_ECUDA", "GSI_EBUSY", "GSI_ISOMORPHISM",
           "GSI_HOMOMORPHISM", "GSI_EDGE_HOST_ONLY", "GSI_ISECT_BSEARCH", "GSI_ISECT_MERGE", "GSI_ISECT_BITMAP"]
