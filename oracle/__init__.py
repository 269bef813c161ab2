"""FP64 CPU oracle for the Spectral Ewald k-space path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` import this package; the product
library (``paper_1712_04732_gb300``) never does, and shares no code with it.

* ``ewald``       -- oracle A: direct Ewald sums (continuum target), plain C.
* ``se_discrete`` -- oracle B: the discrete SE algorithm (Alg. 4) in numpy.
* ``params``      -- the parameter rules of Secs. 3.3, 5, 6.
* ``windows``     -- the window functions of Sec. 4.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
facts fixed outside the oracle (the NaCl Madelung constant, independence of the
total potential from xi, closed-form special cases, library special functions,
quadrature of the defining integrals, numbers printed in the paper).
"""
