"""Seeded synthetic inputs for the cell-based FMM gravity solve.

This package builds octrees of 8x8x8-cell sub-grids (node descriptor arrays) and
density fields sampled at leaf-cell centres.  It holds none of the solver's
arithmetic: no moments, expansions, stencils or forces.  Both the CPU oracle
(``oracle/``) and the CUDA library are fed from here, and nothing here imports
either of them.

Node descriptor rows (int32, 14 columns):
    level, ix, iy, iz, parent, child[0..7], tree_id
Levels start at 1 for the root; a node at level l has integer coordinates in
[0, 2**(l-1)) per axis.  Child k covers the octant (k & 1, (k >> 1) & 1,
(k >> 2) & 1) of its parent.  Leaf nodes have child[*] == -1.  Cells inside a
node are numbered x + 8*y + 64*z.
"""

from .trees import (DESC_COLS, uniform_tree, adaptive_tree, concat_trees,
                    leaf_nodes, leaf_cell_centres, node_cell_width,
                    count_leaves)
from .density import (lane_emden, gaussian_blobs, polytrope_binary,
                      DENSITY_FLOOR)
from .configs import make_config, CONFIG_NAMES

__all__ = [
    "DESC_COLS", "uniform_tree", "adaptive_tree", "concat_trees", "leaf_nodes",
    "leaf_cell_centres", "node_cell_width", "count_leaves", "lane_emden",
    "gaussian_blobs", "polytrope_binary", "DENSITY_FLOOR", "make_config",
    "CONFIG_NAMES",
]
