"""CPU FP64 oracle for the AARMR hot path (arXiv 2205.00385).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library; the only thing both sides use is the seeded problem definitions in
``workloads/``.

Everything here is plain numpy/scipy in float64, written to be checked by eye
against the paper:

* ``fe``          -- element stiffness, grid numbering, assembly, BCs (Eq. 1, 3, 7)
* ``filters``     -- density filter and its transpose (Eq. 31-33)
* ``sensitivity`` -- SIMP modulus, compliance and its derivative (Eq. 1, 4-6, 34)
* ``oc``          -- optimality-criteria update (Eq. 3, method of ref. [31])
* ``solvers``     -- direct solve, PCG, V-cycle multigrid and MGCG (Algorithm 2)
* ``reanalysis``  -- CA, PARM and CARM (Eq. 8-29)
* ``aarmr``       -- the control loop of Algorithm 1 inside the design loop

Functions whose result the paper does not pin beyond their definition say
so in their docstring ("parity unpinned").
"""
