"""CPU oracle for the structure-preserving H^2 matrix-matrix product (Ma & Jiao).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 (complex128
where the kernel is complex) restatement of the method, written to be checked
against the paper by eye.  Only the test-suite, the smoke check and the timed CPU
baseline of the benchmark may import it; the library and its Python binding never
do, and the oracle imports nothing from the CUDA path (it shares only the seeded
input generators, which hold no arithmetic of the method).

Modules:
  tree       cluster tree by cardinality-balanced bisection, block partition by the
             strong admissibility condition (Sec. II, Eq. admCond)
  kernels    kernel functions 1/(4 pi r), 1/r^2, exp(-jkr)/(4 pi r)
  h2         H^2 representation (Sec. II), construction, exact matvec, to_dense
  basis      normalised Gram sum and truncated eigen-decomposition (Sec. III-C, IV-C)
  mmp        the product itself: leaf level (Sec. III), non-leaf levels (Sec. IV),
             top-down split of the coupling matrices held by non-leaf blocks (Sec. IV-E)

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, brute force or special cases (see each module's header).
"""
