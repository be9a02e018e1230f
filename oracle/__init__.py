"""FP64 CPU oracle (test infrastructure only; see oracle.oracle)."""
from .oracle import Oracle, prox_l1, nmse, psnr_magnitude, build, set_threads, get_threads  # noqa: F401
