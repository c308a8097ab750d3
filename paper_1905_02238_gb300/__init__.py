"""GB300-native batched Shannon mutual information (FSMI, Zhang et al., IJRR 2019).

The compute path is the C-ABI library ``libfsmi.so`` (hand-written sm_103a CUDA kernels, sources in
``csrc/``); ``fsmi`` is its thin Python binding. ``synth`` draws the seeded synthetic inputs.
Importing the package loads nothing; the library is loaded on the first call.
"""
