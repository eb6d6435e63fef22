"""GB300-native hot path of the diagonalization-based parallel-in-time method
for fourth-order PDEs (biharmonic heat, linearized and nonlinear
Cahn-Hilliard).  The compute path is libpint (CUDA, sm_103a) behind a C ABI;
``pint`` is its ctypes binding.  Importing the package loads nothing."""
__all__ = ["pint", "synth", "build_lib"]
