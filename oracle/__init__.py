"""CPU oracle for the Krylov return-probability path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg import this package.  The product library never calls it and shares no
code with it: the oracle builds an explicit sorted basis (Algorithm 2), a CSR
Hamiltonian (Sec. 3), runs Arnoldi with full reorthogonalisation (Sec. 2, "Krylov
subspace methods") and a diagonal Pade exponential with Expokit-style time stepping.
Everything is FP64.

Modules:
  basis    -- explicit basis, lookup and CSR Hamiltonian (C, via ctypes)
  pade     -- diagonal Pade exponential with scaling and squaring
  krylov   -- Arnoldi (CGS2) and the time-stepping loop that yields P(t)
  dense    -- dense references for small sectors (Kronecker-product H, eigh, free
              fermions, two-level formula)
  gradient -- dense Daleckii-Krein gradient of P(t) and finite differences
  analysis -- least-squares power-law exponent gamma of C(t) (Sec. 4)
  moments  -- P(t) at early times from the power series of the exponential, for sectors
              too large for the CSR oracle (L = 30)

Parity status of each function is stated in its own docstring ("pinned by ...").
"""
