"""SafeGPU on GB300: contract-checked collections with sm_103a kernels.

Importing the package loads nothing; the CUDA library is loaded by
``paper_1410_6685_gb300.safegpu`` on first use.
"""
