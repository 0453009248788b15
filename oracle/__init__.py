"""FP64 CPU oracle for the per-iteration hot path of density-based inverse homogenization.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute this
package: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
arm use it. It shares no code with the CUDA library (no kernels, headers, tables or
helpers); its only common dependency with the CUDA path is the seeded input generator
module `synthetic`, which holds none of the method's arithmetic.

The oracle is the plain definition of what the method computes, written from the paper
(Zhang et al., arXiv 2301.08911):

* fem.py     - hex8 element matrix, SIMP modulus, periodic assembly, macro-strain loads
               (Eq. 4, Eq. 12), direct solve (Eq. 5), C^H (Eq. 7), sensitivities
               (Eq. 8, Eq. 9), the vertex form of K u (Eq. 13) for sampled vertices.
* filters.py - periodic linear-cone density filter (Sec. 5 material interpolation,
               Sec. 6.4 periodic kernel) and the density-weighted sensitivity filter of
               the unfiltered variant (Sec. 5.3).
* optim.py   - OC volume-constrained update (Sec. 3.3), objectives (Eq. 19-22), one
               whole optimisation iteration.
* init.py    - trigonometric density initialisation with sigmoid projection (Sec. 6.2).
* symmetry.py - orbit averaging under the reflect3 / rotate3 / reflect6 symmetry
               groups (Sec. 6.1).
* learned.py - the warm-start network: periodic 3x3x3 convolutions with their two
               derivatives, forward and backward passes with BF16 rounding points,
               MSE loss and Adam (not part of the paper's method; its readings are in
               the module header).
* pcg.py     - FP64 conjugate gradients preconditioned by block Jacobi or by a symmetric
               V-cycle of mg.py's operators, certified by the true residual of the
               assembled K (the solve of Eq. 5 above the sizes a direct solve reaches).
* mg.py      - explicit trilinear prolongation, Galerkin coarse operators R K I and their
               27-block vertex stencils (Sec. 3.3, Eq. 17-18), 8-colour block Gauss-Seidel
               (Eq. 15-16).

Units: the oracle works in the paper's physical units, Omega = [0,1]^3, h = 1/n,
|Omega| = 1.
"""
from .fem import (  # noqa: F401
    elasticity_matrix,
    ke_hex8,
    element_vertices,
    element_dofs,
    simp_modulus,
    simp_modulus_derivative,
    macro_strain_displacements,
    assemble_K,
    macro_strain_loads,
    solve_cases,
    element_energies,
    homogenized_tensor,
    sensitivity,
    apply_K_at_vertices,
    macro_strain_loads_at_vertices,
    homogenize,
)
from .filters import cone_filter, cone_weights, sensitivity_filter  # noqa: F401
from .symmetry import symmetrize  # noqa: F401
from .init import trig_initialization  # noqa: F401
from .optim import oc_update, objective, optimization_iteration  # noqa: F401
from .mg import (  # noqa: F401
    prolongation,
    galerkin,
    vertex_stencil,
    stencil_matrix,
    gs_sweep,
    level_sizes,
)
