"""GB300-native hp space-time multigrid Newton-Krylov solver for tensor-product space-time
finite elements of the incompressible Navier-Stokes equations (Margenberg & Bause).

The compute path is the C-ABI library libstmg.so (hand-written sm_103a CUDA kernels, see
include/stmg.h); `paper_2602_13841_gb300.stmg` is its thin ctypes binding and
`paper_2602_13841_gb300.inputs` the seeded synthetic input generators.  Importing the package
does not load the library; `stmg.load()` does and raises if it is missing.
"""
