"""Plain, slow FP64 CPU oracle for the IP-GFCC / MOR hot path.

Test infrastructure only: imported by ``tests/``, the package smoke check and the CPU-baseline leg
of the benchmark, never by the CUDA library or its Python binding. It shares no code with the GPU
path; both sides take their inputs from ``synth`` (random numbers and the input recipe only).

Modules: ``fockspace`` (brute-force Fock-space pins), ``hbar`` (similarity-transformed Hamiltonian
elements), ``sigma`` (M x), ``bc`` (b_p, c_q), ``solve`` (dense LU / GMRES, G, A), ``mor``
(subspace, projection, reduced model, adaptive refinement), ``grad`` (adjoint derivatives).
"""
