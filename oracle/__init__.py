"""Exact CPU oracle for colour-coding tree counting (test infrastructure only).

Imported only by the tests, the smoke check and the CPU-baseline leg of the
benchmark; the product path never imports it.
"""
from .oracle import (Result, automorphisms, brute, colourful_probability, count, estimate, py_brute,  # noqa: F401
                     template_csr, weights_to_int)
