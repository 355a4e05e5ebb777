"""GB300-native randomized numerical-rank estimation (Meier & Nakatsukasa).

The compute path lives in ``librankest.so`` (hand-written CUDA for sm_103a behind
a C ABI declared in ``include/rankest.h``); ``rankest`` is its ctypes binding.
Importing this package does not load the library; ``rankest.lib()`` does, and it
raises if the library was not built.
"""
