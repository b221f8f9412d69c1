"""Shared helpers of the GPU parity tests (CUDA library vs CPU oracle)."""
import numpy as np

from workloads import D3Q19_ORDER

C3 = D3Q19_ORDER.astype(np.float64)
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def require_cuda():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_02774_gb300 import build
    build()
    return torch


def pair(case, **kw):
    """GPU Channel and oracle Sim for the same case and parameters."""
    import oracle as O
    from paper_2205_02774_gb300.channel import Channel
    gpu = Channel.from_case(case, **{k: v for k, v in kw.items() if k not in ("oracle_nx",)})
    okw = {k: v for k, v in kw.items() if k not in ("storage", "check_every", "mass_tol", "oracle_nx",
                                                      "use_torch_allocator", "stream", "streaming")}
    if "oracle_nx" in kw:
        c2 = case.with_(nx=kw["oracle_nx"])
        orc = O.Sim.from_case(c2, **okw)
    else:
        orc = O.Sim.from_case(case, **okw)
    return gpu, orc


def velocity(f, F=(0.0, 0.0, 0.0)):
    rho = f.sum(0)
    j = np.einsum("ia,i...->a...", C3, f)
    return (j - 0.5 * np.asarray(F, dtype=np.float64).reshape(3, *([1] * (f.ndim - 1)))) / rho


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def normwise(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def fp16_bits(f64_pops):
    """binary16 bits of f_i - w_i (the shifted FP16 storage format)."""
    h = (f64_pops - W19.reshape(19, *([1] * (f64_pops.ndim - 1)))).astype(np.float16)
    return np.ascontiguousarray(h.view(np.uint16))


def fp16_decode(bits):
    return bits.view(np.float16).astype(np.float64) + W19.reshape(19, *([1] * (bits.ndim - 1)))


def fp16_half_ulp(vals):
    """Half the binary16 spacing at each value (the storage rounding bound)."""
    h = np.abs(vals).astype(np.float16)
    sp = np.spacing(h).astype(np.float64)
    return 0.5 * sp
