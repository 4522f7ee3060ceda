"""B300-native runtime scheduling of small GPU tasks (ACS, arXiv 2401.12377).

``acs``      ctypes binding of libacs.so (the C ABI in include/acs.h)
``harness``  drives seeded task streams through the library
``build``    compiles libacs.so for sm_103a

Importing the package loads nothing; ``acs.load()`` loads the library and
raises if it was not built.
"""
