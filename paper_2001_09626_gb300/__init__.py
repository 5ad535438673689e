"""GB300-native inexact All-Floating IETI solver (arXiv 2001.09626).

The compute path is the CUDA library ``libafieti.so`` (C ABI in
``include/afieti.h``); ``afieti`` is its ctypes binding and ``solver`` adds a
small object wrapper and a torch.autograd.Function for the adjoint."""
from .afieti import *  # noqa: F401,F403
