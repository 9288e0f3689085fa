"""GB300-native SE(2) optimal transport: the log-domain group convolution and the
convolutional Sinkhorn barycenter of arXiv 2402.15322, as a C-ABI CUDA library
(libse2ot.so) with a thin Python binding.

Importing the package loads nothing; `paper_2402_15322_gb300.se2ot` loads the library.
"""
