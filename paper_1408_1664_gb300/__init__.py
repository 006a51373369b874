"""Exact Bayesian-network edge posteriors on GB300 (sm_103a).

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_1408_1664_gb300.binding``.
"""
__all__ = ["binding", "datagen"]
