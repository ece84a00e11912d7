"""GB300-native hull detection for proton CT (SC, MSC, SM).

`paper_1402_1720_gb300.hulld` is the Python binding of the C-ABI library
`libhulld.so` (CUDA kernels for sm_103a); `paper_1402_1720_gb300.synth`
generates seeded synthetic workloads.  Importing this package loads neither.
"""
__all__ = ["hulld", "synth"]
