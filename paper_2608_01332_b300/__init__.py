"""B300-native (sm_103a) rake-compress solver for branched dual-regularized LQR.

The CUDA library ``libtlqr.so`` (C ABI declared in include/tlqr.h) is loaded on
first use by :mod:`paper_2608_01332_b300.tlqr`; importing this package alone
loads nothing.
"""
