"""GB300-native Tile Low-Rank Matérn maximum-likelihood library.

Importing the package is cheap: the CUDA library is loaded on first use by
:mod:`paper_1804_09137_gb300.tlr`, and :mod:`paper_1804_09137_gb300.inputs`
holds the seeded synthetic-input generators (no method arithmetic).
"""
__all__ = ["inputs", "tlr"]
