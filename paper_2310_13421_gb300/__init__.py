"""GB300-native tensorized Pauli decomposition (arXiv:2310.13421).

The CUDA library (``libtpd.so``) is loaded lazily on first use, so that
``paper_2310_13421_gb300.synth`` can be imported without a GPU.
"""
