"""GB300 (sm_103a) implementation of the non-local Variable Eddington Tensor
closure of VETTAM (Menon et al. 2022, arXiv 2202.08778, Sec. 2.2.5).

``vet``   -- Python binding of libvet (the C ABI in include/vet.h)
``synth`` -- seeded synthetic inputs (no method arithmetic)
``build`` -- in-tree nvcc build of libvet for sm_103a
"""
__all__ = ["vet", "synth", "build"]
