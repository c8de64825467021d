"""Plain, slow FP64 CPU oracle of the eigenvector-deflated WaveHoltz method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the `paper_2606_31842_b300`
package, its C-ABI library or its kernels) imports, links or calls this package; only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of
`bench.py` do.  It shares no code with the CUDA path: the only common module is the seeded
input generator `paper_2606_31842_b300.inputs`, which holds no method arithmetic.

Every function is a direct transcription of a definition or algorithm of the paper
(Appelo, Henshaw, Peng, "Numerical study of eigenvector deflation to accelerate the
WaveHoltz method"), cited by section / equation / algorithm, in numpy float64 with no
blocking, fusion or reordering beyond what the definition states.

Modules
  operators   grid, difference operator L_{p,h} (Sec. 2.2, eq. discreteHelmholtz), the
              M = diag(1/c^2) inner product
  waveholtz   time grid, explicit leapfrog + trapezoid filter = Pi_h (eq.
              discreteWaveExplicit, eq. quadrature), S_h, b, A = I - S_h
              (eq. WaveHoltzMatrixEquation)
  spectral    filter transfer beta (eq. beta_fun) and its discrete counterpart beta_h,
              closed-form sine eigenpairs (Sec. 4.3), choice of the deflation set (Sec. 2.3)
  krylov      FPI (Algorithm 1), DEVD (Algorithm 2), CG, DCG (Algorithm 4), GMRES(m)
              (the restarted base of Algorithm 5)
  lanczos     Krylov eigen-solve on S_h (EigenWave idea, Sec. 4.1)
  adjoint     reverse sweep of Pi_h (discrete adjoint of the leapfrog + filter)

Parity pins: see tests/test_oracle_*.py.  Functions without an independent pin say
"parity unpinned" in their docstring.
"""
from . import operators, waveholtz, spectral, krylov  # noqa: F401
