"""GB300 (sm_103a) library for the hot path of the wave-packet
continuum-discretisation Faddeev method (arXiv:1508.07441).

``wpcd``     ctypes binding of the C ABI (include/wpcd.h) to libwpcd.so
``inputs``   seeded synthetic workloads
``build``    in-tree build of libwpcd.so
"""
__all__ = ["wpcd", "inputs", "build"]
