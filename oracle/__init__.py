"""FP64 CPU oracle of the D3Q7 lattice-Boltzmann Maxwell scheme (arXiv 2510.11042).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import anything from this package.  It shares
no code with the CUDA library in paper_2510_11042_gb300/ and never imports it.

Modules:
  lbem_oracle.c  plain C FP64 step (Eqs. 1, 2, 4; TF/SF; absorbing layer; DFT)
  lb.py          ctypes driver: lattice, 1D incident line, DFT window
  ntff.py        near-to-far-field projection (Eqs. 5-10, far-field form)
  mie.py         Lorenz-Mie cylinder/sphere series, exact cylinder near field,
                 current-element fields
  fresnel.py     Eq. 11 and the oblique Fresnel coefficients
  metrics.py     Eqs. 12-13 and the relative-L2 parity metric

Parity status: every function here is pinned by a test in tests/test_oracle_*.py
against values or identities that do not come from the oracle itself.
"""
