"""GB300 implementation of the Roman-Perez--Soler evaluation of the van der
Waals nonlocal correlation energy E_c^nl and potential v_nl.

The compute path lives in ``libvdwnl.so`` (hand-written CUDA for sm_103a,
behind a C ABI declared in ``include/vdwnl.h``); ``vdwnl`` is its thin ctypes
binding and ``autograd`` the torch.autograd.Function built on it.
"""
