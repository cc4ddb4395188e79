"""Plain, slow, FP64 CPU oracle of the method of arXiv 2602.17950.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this package; the product path (the
CUDA library and its Python binding) never does, and shares no code with it.

Contents
  fft    -- own iterative radix-2 FFT (Section 3.2 DFT convention)
  model  -- grid, spectral operators, energy, Hamiltonian, chemical potential,
            spin density, preconditioners (Sections 1, 2.2, 3.2, 3.4)
  pcg    -- Algorithm 1 (PCG), Algorithm 2 (step size), Algorithm 3 (CM-PCG),
            stopping criteria (Sections 3.1, 3.3, 3.4)
  guesses -- initial guesses (a)-(f) of Section 4

Every function states the passage of the paper it follows.  Where the paper is
silent or ambiguous the reading taken is stated in the docstring.
"""
