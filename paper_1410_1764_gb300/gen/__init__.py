"""Kernel generator: symbolic equation lists -> CUDA point bodies.

`python -m paper_1410_1764_gb300.gen` rewrites the generated headers under
csrc/generated/ and the operation counts in csrc/generated/opcounts.json.
"""
