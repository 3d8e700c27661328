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


def rel_inf(a, b):
    """max |a - b| / max |b|: the element-wise error, so that a wrong band of
    cells cannot hide inside a small whole-vector L2 error."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (nb if nb > 0 else 1.0)) if a.size else 0.0


def assert_close(got, ref, tol, what=""):
    """Relative L2 error and element-wise error (relative to max |ref|), both <= tol."""
    e2, ei = rel(got, ref), rel_inf(got, ref)
    assert e2 <= tol and ei <= tol, f"{what} rel L2 {e2:.3e}, rel max {ei:.3e}, bar {tol:.0e}"


# A stopping decision |d| ||y|| <= tol ||p|| can flip between two FP64
# evaluations that differ only by summation order when the quantity lies
# within a few ulps of tol.  A mismatch of iteration counts is accepted only
# for such a borderline stop, and the oracle is then rerun at the GPU's count.
BORDERLINE = 1e-9


def oracle_at_gpu_count(gpu_iters, oracle_iters, forced, tol):
    """Iteration counts of one Leja series, GPU vs oracle.  Returns None when
    they agree (compare with the oracle's own adaptive result).  Otherwise the
    counts must differ by one and the stop must be borderline: ``forced(k)``
    runs the oracle with exactly k iterations and returns (result, err_est),
    err_est being the oracle's stopping quantity |d_k| ||y_k|| / ||p_k||; at
    the smaller count it must lie within BORDERLINE (relative) of tol.  Then
    the oracle's result at the GPU's count is returned, to be held to the same
    bar as equal counts."""
    if gpu_iters == oracle_iters:
        return None
    assert abs(gpu_iters - oracle_iters) == 1, (gpu_iters, oracle_iters)
    _, est = forced(min(gpu_iters, oracle_iters))
    assert abs(est / tol - 1.0) <= BORDERLINE, \
        f"counts {gpu_iters} vs {oracle_iters} with a stopping quantity {est:.6e} not at tol {tol:.1e}"
    ref, _ = forced(gpu_iters)
    return ref
