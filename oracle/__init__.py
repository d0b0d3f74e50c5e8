"""CPU oracle for fixed-radius neighbour search (arXiv 2212.07679).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (``paper_2212_07679_gb300``) never imports, loads or runs it, and
this package imports nothing from the product path.

Contents:

* ``brute_radius``        -- FP64 brute force by direct differences (C, OpenMP);
* ``brute_radius_numpy``  -- the same definition written in numpy (second,
                             independent implementation for small inputs);
* ``pair_dist2``          -- the same definition for sampled (query, point) pairs;
* ``radius_rows``         -- the neighbour lists of selected query rows against a
                             large point set (a float64 product discards the pairs
                             certainly outside; the definition decides the rest);
* ``radius_grid``         -- every query's neighbour list in low dimension, the
                             definition evaluated on pairs of adjacent grid cells;
* ``cpu_snn``             -- Algorithms 1 and 2 in FP64 (plain CPU SNN);
* ``dbscan``              -- DBSCAN on top of the brute-force neighbour lists;
* ``cosine_radius``       -- cosine / angular search by the Euclidean reduction
                             of Section 3 (``normalize_rows`` and the radius
                             mappings);
* ``brute_inner_product`` -- inner-product threshold search (FP64 dot products);
* ``tie_audit``           -- pairs where the FP64 definition's decision differs
                             from exact rational arithmetic (boundary band only).

Pins (tests/test_oracle_*.py): hand cases under tests/golden/, exact
invariants, the paper's printed return ratios (Tables 1 and 2) and the
closed-form distance distribution of the unit square and cube, the Gaussian
blob model of Section 5, and agreement with scipy's FP64 cdist.
"""
from .brute import (brute_radius, brute_radius_numpy, pair_dist2, radius_rows, radius_grid, build_oracle,
                    oracle_threads, CSR)
from .cpu_snn import SNNIndex, snn_index, snn_query, snn_radius
from .dbscan import dbscan, dbscan_bfs
from .cosine import (normalize_rows, radius_for_cosine_distance, radius_for_cosine_similarity,
                     cosine_radius)
from .inner_product import dot_fp64, brute_inner_product
from .tie_audit import tie_audit, exact_is_neighbour

__all__ = ["brute_radius", "brute_radius_numpy", "pair_dist2", "radius_rows", "radius_grid", "build_oracle",
           "oracle_threads", "CSR", "SNNIndex", "snn_index", "snn_query", "snn_radius",
           "dbscan", "dbscan_bfs", "normalize_rows", "radius_for_cosine_distance",
           "radius_for_cosine_similarity", "cosine_radius", "dot_fp64", "brute_inner_product",
           "tie_audit", "exact_is_neighbour"]
