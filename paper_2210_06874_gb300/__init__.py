"""GB300-native (sm_103a) hot path of Hybrid Monte Carlo for the honeycomb
Hubbard model (arXiv:2210.06874, §2): the fermion matrix M[phi] and
M^dagger[phi] with the hopping exponential exp(delta*kappa*h), CG on
M M^dagger, the pseudofermion force, leapfrog and Metropolis.

The compute lives in libhmc_gb300.so (hand-written CUDA, C ABI in
include/hmc.h).  `hmc` is the ctypes binding; `synth` holds the seeded
synthetic inputs; `autograd` wraps the adjoint force as a
torch.autograd.Function.  Importing the package does not load the library;
the first use of `hmc` does, and fails loudly if it has not been built.
"""
__all__ = ["hmc", "synth", "build_lib", "autograd"]
