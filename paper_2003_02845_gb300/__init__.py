"""GB300-native discrete-ordinate neutrino transport step (Chan & Mueller,
arXiv:2003.02845): CUDA kernels for sm_103a behind the C ABI of
include/bt.h, with a thin ctypes binding in ``bt``."""
__all__ = ["bt", "build", "learned_remap", "workloads"]
