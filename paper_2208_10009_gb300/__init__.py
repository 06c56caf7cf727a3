"""GB300 CUDA implementation of the SBR hot path of arXiv 2208.10009 (equiangular ray
launching, BVH tracing with reception, double-count removal, the iterative precise
algorithm, validity test, channel outputs, batched refinement and the unfolding adjoint).

Submodules: ``api`` (Context and handles over the C ABI), ``autograd`` (SbrUnfold),
``scenes`` (seeded synthetic inputs), ``build`` (nvcc build of libsbr.so).
"""
__all__ = ["api", "autograd", "scenes", "build"]
