"""GB300-native AdResS step, force or energy interpolation (sm_103a CUDA behind a C ABI).

Importing the package is cheap: the CUDA library is loaded by
``paper_1806_10841_gb300.adress`` on first use.
"""
