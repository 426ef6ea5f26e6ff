"""GB300-native Gaussian Wave Splatting hot path (arXiv 2505.06582).

``gws`` is the Python binding of the C-ABI library ``libgws`` (CUDA, sm_103a);
``scenes`` draws seeded synthetic inputs.
"""
