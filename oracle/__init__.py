"""FP64 CPU oracle for the demagnetizing-field convolution and the LLG/RK4 step.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain reference that the
CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` -- its CPU-baseline and reference legs, and the error checks it reports
beside the 3D and switching timings -- may import it; the library
(``paper_2308_08447_gb300``) never does, and this package imports nothing from
the library. The two share no code: the library has its own FP64 tensor
generator and FFT, written separately.

Modules
-------
tensor  -- cell-averaged demag tensor N(X, Y, Z) (Sec. II, Eq. 1 and the
           tensor formulas the paper cites), FP64, exact Newell stencil in the
           near field and Gauss-Legendre cell-pair quadrature in the far field.
conv    -- Eq. 1 as a direct O(N^2) sum, and as the zero-padded FFT
           convolution in the step order of Appendix A with a single GPU.
llg     -- exchange field (Eq. 4), the LLG right-hand side (Eq. 5 solved for
           dm/dt) and the classic RK4 step (Sec. III).

Every function works in SI units: metres, A/m, J/m, seconds.
"""
MU0 = 4.0e-7 * 3.141592653589793238462643383279502884
GAMMA = 2.212761569e5  # m/(A s), mu0 * gamma_e
