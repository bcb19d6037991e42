"""GB300-native readout DSP stage of arXiv:1812.02200: polyphase filter bank
and direct multi-tone demodulation behind a C ABI (include/rfr.h).

``paper_1812_02200_gb300.rfr`` is the Python binding (import it after the
library is built; ``paper_1812_02200_gb300.build.build()`` compiles it).
"""
__all__ = ["build"]
