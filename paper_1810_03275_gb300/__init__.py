"""GB300-native (sm_103a) preconditioned primal-dual TV-CT reconstruction with
inequality constraints (PDRQS1).

The compute path lives in the CUDA library ``libctrecon.so`` (built from
``csrc/``) behind the C ABI declared in ``include/ctrecon.h``; ``ctrecon`` is its
thin Python binding.  Importing this package does not load the library; the
first call into ``ctrecon`` does, and fails loudly if it is missing.
"""
__all__ = ["ctrecon", "phantom"]
