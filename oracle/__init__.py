"""Plain, slow, FP64 CPU oracle of the continuous-scale central-moment LBM
(arXiv 1807.02284, Li, Bai, Liu).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library
never calls into it and shares no code with it; the two meet only in the seeded inputs of
``synth``.

Modules
  cmr       lattice, central-moment matrix, equilibrium moments, relaxation rates, collision
  grid      one uniform block: pull-stream, bounce-back, faces, adaptive relaxation, scalar
  coupling  continuous-scale blocks: K-hat rescale, trilinear/temporal interpolation,
            prior-/post-mapping and the Algorithm 1 schedule
  adjoint   FP64 gradients of a smoke-control loss by reverse-mode differentiation of
            ``grid`` (checked itself against central finite differences)

Everything is evaluated with dense 27 x 27 per-node matrices and torch's LU solve in
float64, following the paper's formulas in its own order.
"""
