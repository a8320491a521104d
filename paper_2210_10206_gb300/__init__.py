"""GB300-native SARABANDE hot path: FFT-based 3/4-point correlation functions.

The compute lives in the C-ABI library ``libsarabande_gb300.so`` (CUDA, sm_103a);
``paper_2210_10206_gb300.sbg`` is a thin ctypes binding over it.
"""
