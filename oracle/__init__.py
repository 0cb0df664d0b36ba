"""FP64 CPU oracle of the Yin-Yang direction-splitting AC scheme.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
numpy restatement of the method of "A direction splitting scheme for
Navier-Stokes-Boussinesq system in spherical shell geometries" (arXiv:1905.02300)
written from the paper.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product (the CUDA library and its Python binding) never calls it and shares no
code with it.

Modules:
  grid      -- Yin/Yang geometry, MAC placement, metric (Sec. 2, Sec. 4)
  operators -- discrete rates, divergence, pressure update, 1-D factors
               (Sec. 3.2, Sec. 3.3, Eq. Convect_Douglas, Eq. r_comp/theta_comp/phi_comp)
  linesolve -- Thomas algorithm (Sec. 4)
  exchange  -- Schwarz boundary exchange by interpolation (Sec. 4, Algorithm steps 1, 3, 7)
  scheme    -- the AC step with Schwarz iterations and splitting-error
               reduction (Sec. 3.3, Sec. 4, Eq. er)

Parity status: scheme.Oracle.step at a finite number of Schwarz iterations is
"parity unpinned" as a whole: its exact values are pinned only through the
pieces (operators against continuous operators, line solves against dense LU,
fixed point against a dense solve, convergence orders against manufactured and
closed-form solutions, Yin/Yang congruence).
"""
