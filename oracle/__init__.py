"""CPU oracle for the periodic geometric-multigrid Poisson solve (test infrastructure).

This package is test infrastructure.  Only `tests/`, `__graft_entry__.smoke()`
and the `cpu_baseline` / `--impl reference` legs of `bench.py` may import it.
The CUDA library never calls it, and it shares no code with the CUDA path:
everything here is written from the paper's equations in plain NumPy/SciPy,
float64 throughout, without blocking, fusion or reordering.

Modules
-------
flat   7-point periodic Laplacian, FFT solve, Chebyshev/Jacobi smoothers,
       full-weighting restriction, trilinear prolongation, exact coarsest
       solve, V-cycle and defect-correction solve (Sec. 2.1-2.3, Sec. 3).
curv   moving-mesh geometry (triad, metric, volume element), the conservative
       19-point curvilinear operator, its exact transpose, the curvilinear
       V-cycle, and the adjoint solve with the psi-gradient (Sec. 4.2-4.3,
       Appendix B, Sec. 4.8 adjoint).
grad   4th-order and 2nd-order periodic finite-difference gradients and their
       transposes (Sec. 3 implementation list, Sec. 4.1).

Parity status of each function is stated in its module header.
"""
