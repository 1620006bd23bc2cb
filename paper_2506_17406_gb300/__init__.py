"""GB300-native (sm_103a) solver for the high-order Riesz maps of the de Rham
complex with the orthogonality-promoting basis and interior/interface
preconditioner of arXiv 2506.17406.

``riesz``  -- ctypes binding of ``include/riesz.h`` (libriesz.so)
``inputs`` -- seeded synthetic meshes and right-hand sides
``build``  -- in-tree build of libriesz.so
"""
