"""GB300-native QTT/SFFT homogenisation (SFFT-based Moulinec-Suquet basic scheme).

Importing the package loads nothing compiled; ``paper_2412_11566_gb300.qtt``
binds the CUDA library and fails loudly if it has not been built.
"""
