"""Helpers shared by the GPU parity tests: build a GPU operator and the oracle
operator from the same seeded ``workloads.Problem``.  Expected values always
come from ``oracle``; the CUDA path is only ever the thing under test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operator as oop  # noqa: E402
from oracle import spectral  # noqa: E402

DEV = "cuda:0"


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def ad():
    import paper_2307_12276_gb300 as mod
    return mod


def dev64(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)


def devT(a, precision):
    dt = torch.float64 if precision == 0 else torch.float32
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV).to(dt)


def gpu_operator(p, precision=0, adv_field=None):
    """Operator on the GPU for problem p (fields uploaded as float64)."""
    g = p.grid
    use_field = p.ax_field is not None if adv_field is None else adv_field
    if use_field:
        ax, ay = dev64(p.ax_arr()), dev64(p.ay_arr())
    else:
        ax, ay = float(p.ax), float(p.ay)
    return ad().create_operator(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                                ax, ay, precision)


def oracle_operator(p):
    A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    return A, spectral.gershgorin(A)


def gpu_source(p, precision=0):
    if len(p.source) == 0:
        return None
    return ad().Source([devT(gk, precision) for gk in p.source.g], list(p.source.h))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
