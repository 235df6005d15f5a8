"""GB300 implementation of the SPD HSS preconditioner for SPD H^2 kernel matrices
(Xing, Huang, Chow).  The CUDA library (libspdhss.so) is loaded lazily by ``api``."""

__all__ = ["api", "inputs", "native", "build"]
