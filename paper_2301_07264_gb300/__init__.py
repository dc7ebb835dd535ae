"""GB300-native Monte Carlo Pauli-error trajectory simulator (ArsoNISQ hot path).

The product is the C-ABI library ``libarso.so`` (include/arso.h) built from
``csrc/`` for sm_103a; ``arso`` is its Python binding. Import ``arso``
explicitly: ``from paper_2301_07264_gb300 import arso``.
"""
__all__ = ["arso", "build"]
