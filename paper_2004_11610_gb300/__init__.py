"""GB300-native execution stage of the extra-component method.

The compute path lives in the compiled library libxc (csrc/, C ABI in
include/xc.h); `xc` is its thin ctypes binding.  Importing this package does
not load the library: `from paper_2004_11610_gb300 import xc` does, and raises
if the library has not been built.
"""
