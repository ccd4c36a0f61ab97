"""FP64 CPU oracle for the adaptive GSIS hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow restatement of the method of Zhang, Zeng & Wu,
"adaptive general synthetic iterative scheme" (arXiv 2501.02245): the gas
model of Sec. 2 (Eqs. getmoment, general_model, the reference distributions,
mu_kappa, NSF_constitutive), the GSIS iteration of Sec. 3.1 (kinetic step,
Eq. updatef, Eq. full_constitutive, Eq. macro), the adaptation of Sec. 3.2
(Eq. Kn_Gll, the DVM-region rule, Eq. G13_VDF), the algorithm summary of
Sec. 3.4 and the convergence criterion of Sec. 4.  Beside the monatomic
(Shakhov) path: the reduced distributions of 2D flows (reduced.py), the
two-VDF gas with internal degrees of freedom (rykov.py), and unstructured 2D
meshes with non-uniform velocity grids (unstructured.py, hybrid.py).  Where
the paper defers a detail to other work, the reading taken is stated in the
function that implements it.

Only tests, the smoke entry point and the benchmark's CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding)
never imports, links or executes anything here, and this package imports
nothing from the product.  Every array is float64; velocities are stored with
the x index fastest.
"""
