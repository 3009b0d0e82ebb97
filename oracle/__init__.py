"""Oracle for the EPRL vertex-amplitude shell sum (arXiv:2107.13952).

TEST INFRASTRUCTURE ONLY. A plain, slow CPU restatement of what the paper computes, written
from the paper's equations and used to check the CUDA path. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may
import it; the product package never does, and shares no code, tables or helpers with it.

Modules and the passages they follow:
* ``wigner``     exact {6j}, (3j), 4jm and {15j} (Sec. 2 eq. 15j; Sec. 3 Wigner-symbol library)
* ``dfunc``      SL(2,C) boost matrix elements d^{rho,k}_{jlm}(r) (Sec. 3 eq. francois); their
                 definition is a reading (the paper prints only the structure), pinned by
                 identities in the tests
* ``quadrature`` panelled Gauss rule in x = e^-r (Sec. 3 "Booster coefficients")
* ``booster``    B4^gamma (Sec. 2 eq. booster)
* ``vertex``     A_v by the shell sum (Sec. 2 eq. vertex-ampl; Sec. 3 framed vertex algorithm)
* ``contract``   boundary contraction and its gradients (Sec. 3 usage examples)

Parity status: every function here is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms, symmetries, orthogonality, a brute-force magnetic-number network sum and an
independent quadrature of the defining integral. The vertex amplitude's absolute value is not
printed anywhere in the paper; it is pinned through those component identities.
"""
