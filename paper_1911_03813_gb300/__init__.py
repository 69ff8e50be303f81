"""GB300-native implicit symmetric CP fitting of moment tensors (Sherman & Kolda, arXiv 1911.03813).

The compute path is libstmf.so (hand-written CUDA for sm_103a behind the C ABI in include/stmf.h);
`stmf` is its Python binding and `inputs` holds the seeded synthetic-input generators.
"""

__all__ = ["stmf", "inputs"]
