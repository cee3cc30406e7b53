"""B300-native THPT trace analysis: decode, entry/exit pairing, tally and
timeline of intercepted API traces (the analysis path of THAPI, arxiv
2504.03683) as hand-written sm_103a CUDA behind a C ABI (include/thapi.h).

``thapi`` is the ctypes binding of libthapi.so; ``build`` compiles it.
"""
from . import thapi  # noqa: F401
from .thapi import Context, ThapiError  # noqa: F401
