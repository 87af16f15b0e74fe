"""GB300-native TFHE gate bootstrapping (the hot path under the homomorphic
functional units of arXiv 2101.03403, CryptoEmu).

The compute path is libcryptoemu.so (hand-written sm_103a CUDA behind a C
ABI, include/cryptoemu.h); this package only marshals arguments to it.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import CeError, Context, CloudKey, SecretKey, lib, header_functions  # noqa: F401
