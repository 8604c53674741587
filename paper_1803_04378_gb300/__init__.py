"""GB300-native dense revised simplex (arXiv 1803.04378 method) behind a C ABI.

Import ``paper_1803_04378_gb300.lpgb`` for the ctypes binding of
``include/lpgb.h`` (it loads the built library and fails loudly without it);
``paper_1803_04378_gb300.build`` compiles that library.
"""
