"""Channel workloads, named by what they are and their sizes.

Every case is a Re_tau channel with an STG inlet at x = 0, a zero-gradient
pressure outlet at x = nx - 1, half-way bounce-back walls at the bottom and top
of the y range and periodic z.  Lengths are lattice units; the channel half
height is h = ny / 2.  ``c_smag`` is the coefficient C of nu_t = C delta^2 |S|
(C = Cs^2, so Cs = 0.1 gives C = 0.01).  ``mach_target`` fixes the lattice
velocity scale: the RANS centreline velocity maps to mach_target * c_s.
``t_filter`` is the time constant, in steps, of the first-order filter applied
to the synthetic fluctuations (0 switches it off).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

from .rans_profile import RansProfile, synthetic_rans_profile


@dataclass(frozen=True)
class ChannelCase:
    name: str
    nx: int
    ny: int
    nz: int
    tau0: float = 0.52
    c_smag: float = 0.01
    n_modes: int = 100
    n_fv: int = 48
    re_tau: float = 180.0
    seed: int = 0
    steps: int = 200
    stats_every: int = 10
    t_filter: float = 4.0
    mach_target: float = 0.0516
    storage: str = "fp32"      # "fp32" | "fp16s" (f - w_i stored as binary16) | "fp16sr" (same, stochastic rounding)
    streaming: str = "pull"    # "pull" (two lattices) | "aa" (one lattice updated in place)
    collision: str = "regularized"  # "regularized" | "bgk"
    bc_x: str = "stg"          # "stg" (inlet/outlet) | "periodic"
    bc_y: str = "walls"        # "walls" | "periodic"
    force: tuple = (0.0, 0.0, 0.0)
    beta: float = 2.0
    # sponge zone before the outlet: length in lattice units (0: off), K, p
    sponge_len: float = 0.0
    sponge_K: float = 1000.0
    sponge_p: float = 3.0

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def profile(self) -> RansProfile:
        return synthetic_rans_profile(self.re_tau, self.n_fv, self.beta)

    def with_(self, **kw) -> "ChannelCase":
        return replace(self, **kw)


CASES = {
    # small parity case: 64x32x32, 100 modes, 48 FV cells, 200 steps
    "channel_64x32x32": ChannelCase("channel_64x32x32", 64, 32, 32),
    # production FP32 channel: h = 64, 12h x 2h x 3h, 200 modes, 96 FV cells
    "channel_768x128x192": ChannelCase("channel_768x128x192", 768, 128, 192,
                                       n_modes=200, n_fv=96, steps=20000),
    # mid-size channel (h = 32) used for detailed profiles: 2.4M cells, lattice > L2
    "channel_384x64x96": ChannelCase("channel_384x64x96", 384, 64, 96, n_modes=200, n_fv=96, steps=2000),
    # production cross-section rows (768 x 128) with a shallow span, for detailed profiles: 4.7M cells
    "channel_768x128x48": ChannelCase("channel_768x128x48", 768, 128, 48, n_modes=200, n_fv=96, steps=2000),
    # refined channel: h = 128, 151M cells
    "channel_1536x256x384": ChannelCase("channel_1536x256x384", 1536, 256, 384,
                                        n_modes=200, n_fv=96, steps=20000),
}


def case(name: str, **kw) -> ChannelCase:
    c = CASES[name]
    return c.with_(**kw) if kw else c
