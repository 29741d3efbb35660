"""B300-native generic stencil library: do_all sweeps and do_reduce reductions.

The compute path is ``libgscl.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/gscl.h``); ``binding`` marshals arguments to it.
Importing this package does not load the library; ``binding.lib()`` does, and
fails loudly if it is missing.
"""
