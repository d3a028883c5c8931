"""B300-native hybrid mesh-Gaussian renderer (hot path of arXiv 2506.06988).

The compute path lives in the CUDA shared library ``libhm.so`` built from
``csrc/``; ``paper_2506_06988_b300.lib`` binds its C ABI.  Importing this
package does not load the library: ``lib.load()`` does, and raises if the
library is missing.
"""
__version__ = "0.1.0"
