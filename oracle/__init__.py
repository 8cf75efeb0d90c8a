"""FP64 CPU oracle for the batched lens-equation / source-plane chi^2 path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the library itself never does,
and nothing here imports the library.  Everything is float64 (PyTorch CPU ops,
numpy, scipy.integrate.quad), written straight from the paper's formulas:

* cosmology.py  angular-diameter distances, a_dis = D_ds/D_s (Sec. 1, Sec. 2.1)
* profiles.py   closed forms of alpha and psi_ij per component (Sec. 2.1)
* lensing.py    sums, lens map (Eq. lens_eq), Jacobian (Eq. jac), mu, multi-plane
                recursion (Sec. 2.2), source-plane chi^2 with the analytic source
                (Eq. chi2_src, Sec. 3.1), member scaling relations (Eq. scaling)
* images.py     lens-equation solver: marching squares + segment intersection
                (Sec. 2.3), with an optional Newton polish
* model.py      physical workload descriptions -> lensing units

Parity pins live in tests/test_oracle_*.py.  Functions without an independent
pin say "parity unpinned" in their docstring.
"""
