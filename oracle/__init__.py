"""Plain CPU FP64 oracle for the Riesz-map solver of arXiv 2506.17406.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It restates the paper's construction step by step, in the paper's order and
notation, with no blocking or fusion:

* ``polys``     -- quadrature on the reference simplices and an orthonormal
                   polynomial expansion built by Gram--Schmidt (Arnoldi) on
                   monomials.
* ``refelem``   -- Sections 3-4: bubble spaces, the eigenproblems of
                   Eqs. (3.9)-(3.10), the degrees of freedom of Eqs. (3.14),
                   (3.16), (3.18) and the dual (Ciarlet) basis.
* ``mesh``      -- Section 5 / 6.1: entity enumeration, global DOF numbering
                   and vertex-star patches.
* ``assemble``  -- Eq. (2.8) by quadrature under the pullbacks of Eq. (2.7),
                   CSR assembly, the explicit preconditioner of Eq. (6.11),
                   PCG (Section 7.1) and a sparse direct solve.

Functions that no independent check pins say "parity unpinned" in their
docstring.
"""
