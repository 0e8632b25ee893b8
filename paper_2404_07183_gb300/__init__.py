"""GB300-native (sm_103a) PCF integral matrices.

All-pairs and cross-set L_p distance and L2 Gram matrices of piecewise
constant functions, one merge walk per pair, in hand-written CUDA behind the
C ABI of ``include/pcf.h``.  See ``api`` for the Python binding and
``synth`` for seeded synthetic inputs.
"""
from .api import (PairwiseFn, PairwiseGraph, PcfError, PcfTensors, l2_kernel, parse_metric,  # noqa: F401
                  pcf_check, pcf_cross, pcf_cross_to_host, pcf_pairwise, pcf_pairwise_backward, pcf_pairwise_to_host, pcf_prepare, pcf_segment_integrals, pcf_sort_order,
                  pcf_workspace_size, pdist, pcf_reduce, pcf_combine, mean, std, pairwise, cross,
                  pcf_walk_promoted, pcf_pairwise_weighted, pcf_weighted_workspace_size,
                  pcf_cross_weighted)
from . import abi, build  # noqa: F401
