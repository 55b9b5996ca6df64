"""CPU oracle for the symmetric near-field Schur-complement preconditioned H-matrix EFIE
solve (arXiv 2111.13483).  TEST INFRASTRUCTURE ONLY: imported by tests, by
``__graft_entry__.smoke()`` and by the benchmark's CPU-baseline leg, never by the
solver library or its Python binding.

Plain, slow, complex128 numpy/scipy code that follows the paper step by step:

* ``ordering``  Algorithm 1 with reverse Cuthill-McKee as the bandwidth reducer;
* ``schur``     symbolic fill, the symmetric block Schur elimination of Eqs. 12-21
                (Sec. 3.1-3.2) and the fill-in compression of Sec. 3.4;
* ``krylov``    the transformed system of Eqs. 22-28 and restarted GMRES (Sec. 5);
* ``mie``       the Mie series of a PEC sphere (pins the EFIE inputs, not the method).

It shares no code with the CUDA library.  Every function cites the passage it
follows; what the paper leaves open is fixed as stated in each docstring.
"""
