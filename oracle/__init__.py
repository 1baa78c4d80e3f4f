"""Plain, slow FP64 CPU oracle of the Boltzmann--(ES-)BGK flux-reconstruction stage.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2312_06567_gb300``) never imports it and
shares no code with it: no operators, tables, constants or helpers cross over.

Every function restates one step of the method of Dzanic & Martinelli
(arXiv 2312.06567, "Methodology"), in the paper's notation, with numpy used
only for library primitives (sums, small dense solves).  There is no blocking,
fusion or reordering beyond what the equations state.

Modules
-------
fr        Gauss--Legendre nodes, Lagrange interpolation/derivative, the
          DG-recovering (Radau) correction functions (section "Numerical method").
velocity  Uniform Cartesian velocity grid and trapezoid weights.
mesh      Uniform affine hex box with periodic or Dirichlet faces.
bgk       Moments, primitives, ES temperature tensor, Sutherland law, the
          conservative Newton solve for Q', the F/G equilibrium and source,
          and the ES tensor variant (the discrete Gaussian matching the full
          target stress).
dual      A second, independent route to the Pr=1 discrete Maxwellian
          (convex dual in the exponential parametrisation) used only as a pin.
stage     FR residual with upwind flux and correction lift, SSP-RK3,
          diagnostics (totals, entropy, L2).
curved    FR on curvilinear hexahedra (GLL curl-form metric terms, transformed
          flux), diffuse walls and collapsed faces.
diagnostics  Macroscopic fields, the local mean free path and Kn_GLL (FR
          density gradient; box and curvilinear meshes, section "Results").
mlp       FP64 forward/backward of the small SiLU network used for the
          learned Q' initial guess.
"""
