"""Plain, slow, complex128 CPU oracle for the CVS-ADC(2) hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import anything under ``oracle/``.  The
product path (the C-ABI library and its Python binding) never imports,
links or calls it, and shares no code with it.

Modules:

* ``integrals`` -- explicit antisymmetrised integrals from Cholesky vectors;
* ``mp2``       -- MP2 doubles amplitudes, MP2 energy, MP2 vv density (Eq. 15);
* ``fns``       -- frozen natural spinors (Eqs. 17-20) and B^P rotation;
* ``adc2``      -- CVS spaces and packing, explicit CVS-ADC(2) blocks,
                   matrix-free sigma, transition moments, eigen-solvers;
* ``fci``       -- determinant-space engine and brute-force ISR, the
                   independent pin of the ``adc2`` element formulas;
* ``spectrum``  -- Lorentzian-broadened spectrum from roots and oscillator
                   strengths;
* ``cisd``      -- CIS(D) energies and the frozen-natural-spinor correction
                   of Eqs. 21-22;
* ``rootsel``   -- canonical CIS guesses mapped into the FNS basis and
                   root-specific selection of the CVS-ADC(2) roots;
* ``grad``      -- the gradient of a sum of roots with respect to the spinor
                   energies and the Cholesky vectors, by torch autograd of
                   the explicit matrix (CPU, complex128), pinned by central
                   differences of ``adc2`` eigenvalues.

Parity status of each function is stated in its docstring.  The modified
transition moments are pinned by the brute-force ISR through second order:
F^(0) and F^(1) for all CVS rows, and the second-order singles term F^(2)_S
(``adc2.transition_moments(..., order=2)``) together with the second-order
ground-state amplitudes it is built from.
"""
