"""CPU oracle (test infrastructure only): see h2ulv_oracle.py."""
from .h2ulv_oracle import (Problem, H2Operator, ULVFactor, refine, kernel_matrix,
                           cluster_tree, interaction_lists, top_level, far_samples,
                           pivoted_qr, pivoted_cholesky, interpolation_matrix, fold_rows)
