"""matgraph for GB300: batched periodic cutoff / KNN multigraphs of crystal structures
(arXiv 2307.05380) with differentiable edge vectors, as hand-written CUDA for sm_103a
behind a small C-ABI (include/matgraph.h).

Python here marshals arguments only; importing works without a GPU, while every call
that computes needs the CUDA library (no CPU fallback).
"""
from .graph import (Batch, EdgeVectors, Graph, Step, autotune, autotune_cached, set_tuned_table, tuned_table, build_per_structure, context, cutoff_graph,
                    cutoff_graph_atoms, edge_vectors, edge_vectors_bwd, edge_vectors_fwd, graph_to_host,
                    host_buffers, knn_graph, last_launch_count, make_opts, measure_fp_peaks, profile_enable,
                    rebuild, stage_times, symmetrize, triplets, update_graph)
from ._build import build as build_library

__all__ = ["Batch", "Graph", "EdgeVectors", "cutoff_graph", "cutoff_graph_atoms", "knn_graph", "update_graph",
           "rebuild", "build_per_structure", "edge_vectors", "edge_vectors_fwd", "edge_vectors_bwd", "autotune",
           "context", "last_launch_count", "make_opts", "build_library", "profile_enable", "stage_times",
           "symmetrize", "triplets", "graph_to_host", "host_buffers", "measure_fp_peaks",
           "Step", "autotune_cached", "tuned_table", "set_tuned_table"]
