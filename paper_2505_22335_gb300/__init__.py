"""GB300-native (sm_103a) differentiable render path of anchor-decoded 3D Gaussians.

The compute lives in a C-ABI CUDA library (``csrc/``); ``binding`` loads it
with ctypes and passes plain device pointers.  ``scenes`` draws seeded
synthetic inputs.  Importing the package does not load the library; the first
call into ``binding`` does, and raises if it has not been built.
"""
