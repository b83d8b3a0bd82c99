"""B300-native analytic-PSF Gaussian slice-to-volume forward model and adjoint.

The compute path lives in the CUDA library ``libgsvr.so`` (sources in
``csrc/``), reached through the ctypes binding in ``gsvr.py``.  Importing the
package itself loads nothing; ``from paper_2512_11624_b300 import gsvr`` loads
the library and raises if it is missing.
"""
