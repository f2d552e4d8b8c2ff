"""GB300-native (sm_103a) BLINK dirty-image library.

The compute lives in ``libblink.so`` (CUDA, C ABI declared in
``include/blink.h``); :mod:`paper_2405_13478_gb300.binding` marshals
PyTorch tensors into it.  Importing this package does not load the library;
``binding.lib()`` does, and raises if it has not been built.
"""

__all__ = ["binding", "build"]
