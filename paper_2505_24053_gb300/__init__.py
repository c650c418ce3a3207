"""GB300-native exact ray-Gaussian renderer (3DGEER, arXiv 2505.24053).

The CUDA library is loaded on first use (see `geer.lib()`); importing the package
alone does not touch the GPU.
"""
