"""GB300-native well-balanced WCSPH hot path (sm_103a CUDA behind a C-ABI).

The CUDA library is loaded lazily by :mod:`paper_2608_22269_gb300.wbsph`;
importing the package itself loads nothing, so that the input generators in
:mod:`paper_2608_22269_gb300.scenes` can be used without a GPU.
"""
__all__ = ["scenes", "wbsph"]
