"""GB300-native orbit-reduced QAOA MaxCut energy and adjoint gradient.

Importing the package loads nothing; the CUDA library is opened on first use
by :mod:`paper_2101_10296_gb300.qaoa`.
"""
