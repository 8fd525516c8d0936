"""FP64 CPU oracle for the Floquet spin-chain evolution.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  product_state   pinned: closed-form single-site expectations, norm
  expm_herm       pinned: scipy.linalg.expm, unitarity, closed form for X
  apply_2q / 1q   pinned: dense Kronecker-product operators (L <= 8)
  period/evolve   pinned: dense exponentials of each layer (L <= 10), J = 0
                  closed-form precession, norm and echo invariants,
                  reflection symmetry, brute force at L = 2, 3
  energy          pinned: dense <psi|H0|psi>, product-state closed form
  adjoint         pinned: central finite differences of the oracle's own
                  forward evolution (and the dense forward evolution)
"""
