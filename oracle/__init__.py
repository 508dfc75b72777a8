"""FP64 CPU oracle for the matrix-free DG time-domain Maxwell right-hand side.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this package; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle computes the plain definition of the semi-discrete DG system of
Kapidani & Schoeberl (arXiv 2002.08733), Sec. II-IV, by assembling every
element's mass, volume-curl and face-coupling matrices with quadrature in
physical coordinates, and then time-stepping the assembled system.  It uses
none of the identities the GPU path relies on (geometry-free reference curl,
Eq. (matrix_free_curl); Piola map, Eq. (piola_transf); the at-most 3x3
block mass structure; sorted-vertex face alignment); those identities are
*checked* by the oracle's tests instead.

Modules
-------
basis     Jacobi polynomials, the orthonormal Dubiner basis (Sec. II,
          Eq. (dubiner_functions)/(ortho_cond)), collapsed quadrature.
mesh      element maps (Eq. (mapping_template)), geometric face matching.
assemble  element and global matrices of Eqs. (uwc), (cwc) plus an upwind
          generalisation, PEC walls, PML mass terms (Sec. IV).
solver    right-hand side, LSRK4 and leapfrog stepping, projection, energy,
          point sources and receivers.
"""
