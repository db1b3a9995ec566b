"""GB300-native explicit step of the all-regime, well-balanced acoustic-transport
scheme (Padioleau et al., arXiv:1903.09043), behind a C-ABI CUDA library.

``paper_1903_09043_gb300.ark`` is the thin ctypes binding of ``libark.so``;
``paper_1903_09043_gb300.inputs`` builds seeded synthetic initial data.
"""
