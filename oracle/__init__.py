"""CPU oracle for the shifted-Green-function, FFT-accelerated Nystrom method (Bruno & Maas).

TEST INFRASTRUCTURE ONLY. Plain, slow, FP64 numpy/scipy code that restates the paper's
definitions and algorithms in its own order and notation. Only `tests/`, `__graft_entry__.smoke()`
and the `cpu_baseline` / `--impl reference` legs of `bench.py` may import it. The CUDA library never
uses it and it shares no code with the library; the two meet only through the seeded inputs of
`paper_1707_04950_gb300.inputs`.

Modules
  green   free-space G, shifted G_j, windows, shifted spectral series, windowed lattice sums (Sec. 2-3)
  direct  the exact Nystrom system (1/2 I + D^dx) mu = -u^inc and Rayleigh extraction (Sec. 2, 4)
  accel   the accelerated forward map, Algorithm 2 (initialisation) and Algorithm 3 (Sec. 5);
          Accel.field: Algorithm 3 at targets off the surface
  field   the scattered field off the surface by its definition (eq. int_eq_dirichlet discretised)
          and by its Rayleigh form above every node; gradient: derivatives of e_n by definition

Parity status: every function is pinned by tests/test_oracle_*.py (closed forms, identities,
brute force, energy balance, and the energy-balance errors the paper prints for its composite and
sinusoid tables, tests/golden/) except the exact values of B_n for curved surfaces, which the paper
does not print ("parity unpinned" for those values; only energy balance and invariances fix them).
"""
