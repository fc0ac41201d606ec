"""FP64 CPU oracle of the per-cell reaction step -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct NumPy code (float64 throughout) that the CUDA path is
checked against. It shares no code, constants table or helper with the CUDA library and
never imports it. Only the tests, the smoke check of ``__graft_entry__`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never calls it.

What the paper fixes and what it leaves open:
  * Sec. 2 (Deep learning approaches): the chemistry network takes (T, p, Y_i) and yields
    the chemical change; real-fluid properties follow the Peng-Robinson EoS.
  * Sec. 3.3.1: inputs are Z-score normalised; everything but the network is double.
  * Sec. 3.3.2: GELU in its tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
  * Silent (textbook readings): the Peng-Robinson equations (Peng & Robinson 1976) with
    van der Waals mixing and k_ij, NASA-7 ideal-gas thermo, Box-Cox transform
    (Box & Cox 1964), Newton recovery of T from conserved enthalpy, mass-action kinetics.

Modules: thermo (NASA-7), pr_eos (Peng-Robinson), network (Box-Cox, normalisation, GELU,
MLP, its Jacobian), step (active-cell list, reaction step, real-fluid properties, T from h,
finite-difference Jacobian of the step), truth (the stiff-chemistry ground truth the network
stands in for: C, BDF, oracle/truth.c), solver (the sparse kernels of Sec. 3.2: LDU matrix,
SpMV, block Gauss-Seidel, finite-volume Laplacian), propnet (the PRNet-style property network:
inputs, outputs, exact properties).
"""
from . import thermo, pr_eos, network, step, solver, propnet  # noqa: F401
