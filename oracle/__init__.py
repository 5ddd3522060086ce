"""CPU oracle for the TTN-TDVP hot path of the Rydberg digital twin (arXiv 2210.03763).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (``paper_2210_03763_gb300/csrc``): separate tree builder,
separate Hilbert-curve code, separate QR, Krylov and contraction code.

Plain, slow, complex128 NumPy/SciPy.  Two parts:

* ``exact``  -- Oracle-X, exact state-vector propagation of the Rydberg
  Hamiltonian (Eq. 1 with the pair term of Eq. 2) for at most 9 atoms.
* ``ttn``    -- Oracle-T, the single-site TTN-TDVP of Sec. "Tensor network
  simulations", step by step, in plain tensordot contractions.
* ``adjoint`` -- the gradient of the final-state fidelity in piecewise-constant
  pulse amplitudes, by exact reverse mode on the state vector (<= 6 atoms).

Pins (values fixed by something other than this code) live in
``tests/test_oracle_*.py``.  Functions without a pin say "parity unpinned" in
their docstring.
"""
