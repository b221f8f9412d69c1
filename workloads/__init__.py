"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

Nothing in this package performs any step of the STG-LBM method. It only
produces the *inputs* the method starts from:

* a closed-form stand-in for the RANS solution at the interface (the paper
  obtains it from a k-omega finite-volume solve, Sec. IV; that solver is not
  part of this project), laid out on a tanh-stretched finite-volume grid;
* the channel workloads (lattice sizes, relaxation time, mode counts) used by
  the tests and the benchmark;
* seeded random population fields used to start parity checks from an
  identical state.
"""
from .rans_profile import RansProfile, synthetic_rans_profile, tanh_grid  # noqa: F401
from .configs import ChannelCase, CASES, case  # noqa: F401
from .states import perturbed_equilibrium_field, D3Q19_ORDER  # noqa: F401
