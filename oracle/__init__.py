"""CPU oracle for the LRBMS two-phase flow method (test infrastructure only).

This package is a plain, slow, FP64 NumPy/SciPy restatement of the paper's
schemes, used to check the GPU library. Only the test suite, the smoke check
and the CPU-baseline leg of the benchmark may import it; the library never
does, and it imports nothing from the library.

Modules, each following the passage named in its docstring:
  grid       fine Cartesian grid, faces, coarse subdomains (Sections 3.1, 4.2)
  physics    mobilities, fractional flow (Eqs. brooksCorey, frationalFlow)
  swip       SWIP-DG pressure bilinear/linear forms (Eqs. swipBilP,
             penaltyParam, Remark 1, linear form l_h, Definition 1)
  velocity   conservative total-velocity reconstruction (Definition 2)
  transport  upwind saturation update for piecewise constants (Definition 3,
             Eq. upwind) and the CFL time step
  impes      high-dimensional two-phase scheme (Algorithm 1)
  tof        time-of-flight (Eq. timeOfFlight)
  offline    mobility profiles, least-squares fit, basis construction and
             offline/online decomposition (Eqs. parameterizedMob,
             leastSquaresFit, Algorithm 2, Section 4.4)
  reduced    LRBMS online time step (Algorithm 3, step 5; Eq. reducedSystem)

Parity status: every function is pinned by a test under tests/ against closed
forms, invariants, brute force or library routines, except the choice of
mean weights on faces (reading R3), which no closed form distinguishes.
"""
