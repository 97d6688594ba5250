"""FP64 CPU oracle for the MacLAB step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import anything here.  The CUDA library and its Python
binding never do, and nothing here imports them.

* ``oracle.py`` / ``maclab_oracle.c``: the plain FP64 MacLAB step (Eqs. (2),
  (4), (5), walls and periodic wrap), its adjoint, unit maps, diagnostics.
* ``lbm_tau1.py``: an independent stream-and-collide LBM, Eq. (1), used to pin
  the oracle through the tau = 1 reduction of the Methods section.
* ``exact_rational.py``: exact rational brute force on tiny grids.
"""
