"""CPU oracle for the one-shot Parareal topology-optimisation pass (arXiv 2411.19030).

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 NumPy/SciPy code that restates the
paper's method step by step.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The CUDA
product path never imports, links or calls anything here, and this package never
imports the product package: the two share no code.

Modules
-------
``fem``        Sec. 2.1-2.2: SIMP interpolation (Eq. 2.5-2.6), Galerkin bilinear
               element matrices by Gauss quadrature, global K, C and load vectors.
``stepping``   Sec. 2.2 and 4.1: backward Euler (Eq. 2.7), the power-mean objective
               (Eq. 2.11), the discrete adjoint (Eq. 4.4-4.7) and the sequential pass.
               Each linear solve is a direct factorisation (factored once per matrix) and
               its triangular solves: banded Cholesky, or a sparse LU on grids whose band is
               wider than 300 nodes.
``parareal``   Sec. 4.2-4.4, Algorithms 1-3: the propagators H, F, G, the modified
               (history-storing) forward Parareal, the reverse vanilla Parareal, the
               k-iteration scheme, the one-shot pass and the PLT variant (Sec. 7).
``allatonce``  Eq. 2.8-2.9 and 4.3: dense brute-force space-time solves, used only on
               tiny grids as an independent check of the time-stepping recursions.
``design``     Sec. 2.1 and 3: the density filter, the threshold projection, the area
               constraint, their chain rule, and the Method of Moving Asymptotes (Svanberg's
               1987 method, one constraint) of the design update in Alg. 3.
``coarse_mesh`` Sec. 7.3 (future work): coarse propagators on the mesh of spacing 2h
               (averaged design, injection and bilinear interpolation between the meshes).

Pins (``tests/test_oracle_*.py``, run with ``-m "not gpu"``): the separable-eigenmode
closed form, the discrete energy balance, the dense all-at-once solve, central
finite differences of the gradient, Parareal's exactness after N_tau iterations,
the M = 1 and N_tau = 1 degenerate cases, the coarse propagators G_pri and G_adj at M > 1
chained over every slice against the sequential primal and adjoint passes of the coarsened
problem (Ntau steps of dtau, loads at the coarse points), the one-shot fixed point, mirror symmetry,
the constant-field objective identity, the homogeneity of Theta in q, and the adjoint
propagators' affinity in the state and linearity in the source scale (Eq. 4.6-4.7); for the
modified objective of Sec. 7.1, Theta~ = Theta^p and the gradient identity
grad Theta = Theta^(1-p)/p grad Theta~; for PLT (G = 0, Sec. 7), its fixed point and its
exactness after N_tau iterations; for the design update, the filter's averaging and its
reproduction of affine fields, the projection's fixed points and derivative, central
differences through filter, projection and objective, and MMA on problems with closed-form
optima; for the coarse-mesh propagators, bilinear reproduction by the interpolation,
the restricted load and the Galerkin products against the operators assembled on 2h,
Galerkin orthogonality of a coarse step, the one-shot fixed point, exactness after N_tau
iterations, and second-order agreement with the fine-mesh coarse step.
The one-shot estimate for a design that differs from the warm-start design is pinned in
closed form where the problem reduces to scalars: uniform designs, no load, Dirichlet sinks on
the whole boundary and a sine mode, with the old design's exact states as the warm start.
There every state is a multiple of the mode, and T, Theta~, lambda and the gradient of the pass
(p = 2 for the adjoint half) are explicit sums over the slices; planted mistakes in the
propagators fail them.  The same reduction pins the coarse-mesh propagators and k-iteration
Parareal (the binomial iterates of Gander and Vandewalle, 2007; the reverse iterations in
matrix form).  For a non-uniform design there is no closed form: beyond the fixed point the
same code runs unpinned.
"""
from .fem import Material, Problem, element_matrices, simp, assemble
from .stepping import (Operator, objective, objective_from_modified, sequential_primal, sequential_adjoint,
                       sequential_pass, sensitivity_term)
from .parareal import (F_pri, G_pri, F_adj, G_adj, oneshot_pass, parareal, coarse_states_from_sequential)

__all__ = [
    "Material", "Problem", "element_matrices", "simp", "assemble",
    "Operator", "objective", "objective_from_modified", "sequential_primal", "sequential_adjoint", "sequential_pass", "sensitivity_term",
    "F_pri", "G_pri", "F_adj", "G_adj", "oneshot_pass", "parareal", "coarse_states_from_sequential",
]
