"""GB300-native BLDTT compute phase (barycentric Lagrange dual tree traversal).

The CUDA library sits behind the C ABI declared in include/bldtt.h; the
Python binding (``paper_2012_06925_gb300.binding``) only marshals arguments.
Import the binding explicitly; importing the package itself loads nothing.
"""
