"""GB300-native DNN-MG hot path: libdnnmg (CUDA, sm_103a) and its binding."""
from . import dnnmg  # noqa: F401
