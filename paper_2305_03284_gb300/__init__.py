"""GB300-native Dynamic DH-MBIR (arXiv:2305.03284): per-frame EM step in libddh (sm_103a).

``from paper_2305_03284_gb300 import ddh`` loads the binding (torch + libddh.so).
"""
__all__ = ["ddh", "build"]
