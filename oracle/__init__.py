"""FP64 CPU oracle (test infrastructure only; see oracle.oracle)."""
from .oracle import (Oracle, prox_l1, prox_group, voxel_groups, group_norms, nmse, psnr_magnitude, build,  # noqa: F401
                     set_threads, get_threads)
