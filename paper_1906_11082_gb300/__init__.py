"""GB300 filtered-Lanczos normal-mode solver (arXiv 1906.11082 hot path).

The compute lives in libnm.so (CUDA for sm_103a, C ABI in include/nm.h);
``paper_1906_11082_gb300.nm`` is its thin Python binding and raises on
import when the library is missing (there is no CPU fallback).
"""
