"""CPU oracle for the EREM / real-Leja phi_1 path of arXiv 1209.5553.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` (its ``cpu_baseline`` object and its
``--impl reference`` arm) may import this package.  The product package never
imports it, shares no code with it, and fails loudly when its CUDA library is
missing instead of falling back to anything here.

It is a plain, slow FP64 restatement of what the paper computes, written in
numpy / scipy (sparse matrix-vector products, a dense matrix product, sparse
LU solves and FFT-free arithmetic serve as library steps):

* ``oracle.fv``        space discretization of §2 and §3.1 (pressure system,
                       Darcy fluxes, heat right-hand side G and its Jacobian J)
* ``oracle.leja``      Gershgorin interval, Leja points (eq. ``lejaa``),
                       divided differences by the matrix function (§4.2),
                       Newton form with error estimate and stopping rule
                       (eq. ``newt``, §4.2)
* ``oracle.krylov``    Arnoldi / modified Gram-Schmidt (Algorithm ``alg:al2``),
                       the phi_1 approximation of eq. ``approphi`` (§4.1) with
                       error estimate and substeps
* ``oracle.adjoint``   gradients of a temperature misfit with respect to T^0
                       and ln K through frozen-schedule EREM steps (transposed
                       Newton polynomial, face-flux and pressure adjoints)
* ``oracle.nonauto``   non-autonomous EREM (eq. ``nEERMg``): phi_1 and phi_2
                       by Leja interpolation, D_t G of a time-dependent
                       inflow temperature
* ``oracle.timestep``  EREM (eq. ``EERM``), ROSM (eq. ``ROS``), ROS2(1)
                       (eq. ``ROSMh``, Table ``ros2``), pressure solves and the
                       sequential coupling of §3.2

Every function is pinned by ``tests/test_oracle_*.py`` against something
other than itself: closed forms, dense matrix exponentials, high-precision
divided differences, brute force on tiny inputs, conservation laws and the
constants the paper prints (``tests/golden/``).
"""
from . import adjoint, fv, krylov, leja, nonauto, timestep  # noqa: F401
from .fv import Grid, Physics  # noqa: F401
from .leja import LejaOptions, LejaResult, phi1_leja  # noqa: F401
