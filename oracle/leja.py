"""Leja-point interpolation of exp and phi_1 (oracle), Section 2 of the paper.

Method (Section 2, the paragraph after Eq. exp_quad_Gauss, and the recurrence
printed below it):
  * alpha is an estimate of the largest-magnitude (negative real) eigenvalue
    of A; the smallest is taken as 0;
  * c = alpha / 2 and gamma = -alpha / 4 map [alpha, 0] onto the Leja interval
    [-2, 2]: z = c + gamma xi;
  * f(xi) = exp((c + gamma xi) dt) or phi_1((c + gamma xi) dt) is interpolated
    at Leja points xi_0, xi_1, ... with Newton divided differences d_m;
  * the Newton form is evaluated on the matrix by
        y_{m+1} = ((A - c I) / gamma - xi_m I) y_m ,  p_{m+1} = p_m + d_{m+1} y_{m+1},
    starting from y_0 = v, p_0 = d_0 v.

Readings where the paper is silent (each is listed in the design notes):
  * Leja points: xi_0 = +2 (so z = 0 is a node), then greedily
    xi_k = argmax_{xi in [-2, 2]} prod_{j<k} |xi - xi_j|; the maximiser in each
    gap between existing points is the root of sum_j 1/(xi - xi_j), found to
    full precision; ties (relative 1e-12 in the log-product) go to the larger xi.
  * Stopping rule: after term m+1 (m+1 >= 2), stop when
        |d_{m+1}| ||y_{m+1}||_2 <= tol ||p_{m+1}||_2 ;
    fail (not converged) after ``max_iters`` terms, or at once when either
    norm is not finite (NaN input, or terms that overflow because the bound
    leaves part of the spectrum far outside the interpolation interval).  ``force_iters`` runs an
    exact number of terms with no test.
  * Substepping: if rho = gamma dt exceeds rho_max, the step is split into K
    equal substeps (K = ceil(rho / rho_max)).
  * Adaptive substeps (optional; the paper fixes no control): start from the
    substep of the rule above; a substep whose series reaches the iteration
    budget max_iters without meeting the stopping rule is rejected and retried
    at half the size; after an accepted substep of m iterations the next one
    doubles when 4 m <= max_iters and the previous attempt was not rejected;
    the last substep is the remainder of the step.  More than MAX_REJECTS
    rejections or MAX_SUBSTEPS accepted substeps give up (not converged, input
    returned unchanged).

Pins (tests/test_oracle_leja.py): first Leja points in closed form and the
greedy-max invariant on a dense grid; divided differences reproduce f at the
nodes and are exact for polynomials; the scalar 1x1 run reproduces
phi_1(z) = expm1(z)/z; dense-matrix runs reproduce scipy's expm of the
augmented matrix.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from functools import lru_cache

import numpy as np

MAX_ITERS = 500
MAX_REJECTS = 40
MAX_SUBSTEPS = 4096


@lru_cache(maxsize=4)
def leja_points(n: int) -> np.ndarray:
    """First ``n`` Leja points on [-2, 2] (reading above; Section 2 cites Caliari04).

    In each gap (a, b) between sorted existing points the log-product has one
    maximiser, the root of sum_j 1/(xi - xi_j).  Multiplying by (xi-a)(xi-b)
    gives the smooth increasing function
        q(xi) = (xi - a) + (xi - b) + (xi - a)(xi - b) sum_{j: xi_j not in {a, b}} 1/(xi - xi_j),
    q(a) = a - b < 0 < q(b) = b - a, solved by bracketed Newton to full precision.
    """
    pts = [2.0]
    if n > 1:
        pts.append(-2.0)
    while len(pts) < n:
        p = np.array(pts)
        s = np.sort(p)
        a, b = s[:-1], s[1:]
        lo, hi = a.copy(), b.copy()
        x = 0.5 * (a + b)
        other = (p[None, :] != a[:, None]) & (p[None, :] != b[:, None])
        done = np.zeros(len(x), dtype=bool)
        for _ in range(200):
            inv = np.where(other, 1.0 / (x[:, None] - p[None, :]), 0.0)
            R = inv.sum(axis=1)
            Rp = -(inv * inv).sum(axis=1)
            q = (x - a) + (x - b) + (x - a) * (x - b) * R
            qp = 2.0 + (2.0 * x - a - b) * R + (x - a) * (x - b) * Rp
            step = q / qp
            conv = np.abs(step) <= 2e-16 * np.maximum(1.0, np.abs(x))
            lo = np.where(q < 0, x, lo)
            hi = np.where(q < 0, hi, x)
            xn = x - step
            bad = (xn <= lo) | (xn >= hi) | ~np.isfinite(xn)
            xn = np.where(bad, 0.5 * (lo + hi), xn)
            x = np.where(done | conv, x, xn)
            done |= conv
            if done.all():
                break
        v = np.log(np.abs(x[:, None] - p[None, :])).sum(axis=1)
        best = v.max()
        cand = np.nonzero(v >= best - 1e-12 * max(1.0, abs(best)))[0]
        pts.append(float(x[cand].max()))
    return np.array(pts)


def divided_differences(x: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Newton divided differences d_m = f[x_0, ..., x_m] (textbook recurrence)."""
    d = np.array(f, dtype=np.float64, copy=True)
    n = len(x)
    for j in range(1, n):
        d[j:] = (d[j:] - d[j - 1:-1]) / (x[j:] - x[:n - j])
    return d


def phi1_scalar(z):
    """phi_1(z) = (e^z - 1)/z with phi_1(0) = 1 (Section 2, recursion from phi_0 = exp)."""
    z = np.asarray(z, dtype=np.float64)
    small = np.abs(z) < 1e-8
    zs = np.where(small, 1.0, z)
    return np.where(small, 1.0 + z / 2.0 + z * z / 6.0, np.expm1(zs) / zs)


def phi_l_scalar(z: float, l: int) -> float:
    """phi_l by the recursion phi_{l+1}(z) = (phi_l(z) - 1/l!)/z, for |z| not tiny;
    the Taylor series sum_k z^k / (k + l)! otherwise."""
    if abs(z) < 0.5:
        return float(sum(z ** k / math.factorial(k + l) for k in range(30)))
    v = math.exp(z)
    for k in range(l):
        v = (v - 1.0 / math.factorial(k)) / z
    return v


def shift_scale(alpha: float):
    """c = alpha/2, gamma = -alpha/4 (Section 2)."""
    return alpha / 2.0, -alpha / 4.0


@dataclass
class LejaStats:
    iters: int = 0          # Leja iterations (matrix-vector products inside the series)
    matvecs: int = 0        # all matrix-vector products
    substeps: int = 1       # accepted substeps
    err_est: float = 0.0
    converged: bool = True
    rejected: int = 0       # adaptive substeps rejected
    sizes: tuple = ()       # accepted substep sizes (adaptive control)


def n_substeps(alpha: float, dt: float, rho_max: float) -> int:
    c, gamma = shift_scale(alpha)
    rho = gamma * dt
    return max(1, int(math.ceil(rho / rho_max))) if rho > rho_max else 1


def adaptive_substeps(dt: float, K0: int, budget: int, attempt):
    """The adaptive substep rule of the module docstring.

    ``attempt(h)`` runs one series of substep size h from the current state and
    returns (ok, iterations); the caller keeps the attempt's result and commits
    it when the next call is made or the rule returns.  Returns
    (sizes, rejected, ok, accepted_flags) where accepted_flags lists, per
    attempt, whether it was accepted.
    """
    h = dt / K0
    done = 0.0
    rejected = 0
    grow = True
    sizes = []
    flags = []
    while True:
        rem = dt - done
        last = h >= rem or rem - h <= 1e-12 * dt
        hs = rem if last else h
        ok, it = attempt(hs)
        flags.append(bool(ok))
        if not ok:
            rejected += 1
            if rejected > MAX_REJECTS:
                return sizes, rejected, False, flags
            h = hs / 2.0
            grow = False
            continue
        sizes.append(hs)
        done += hs
        if last:
            return sizes, rejected, True, flags
        if len(sizes) >= MAX_SUBSTEPS:
            return sizes, rejected, False, flags
        h = 2.0 * hs if (grow and 4 * it <= budget) else hs
        grow = True


def _newton_series(matvec_shifted, y0, d, xi, tol, force_iters, max_iters, top=None):
    """Evaluate sum_m d_m y_m with y_{m+1} = (X - xi_m) y_m (X = (A - c)/gamma).

    ``matvec_shifted(y, m)`` returns X y (plus the augmented coupling for
    iteration m).  ``top`` selects the part of the vector used for the norms.
    Returns (p, iterations, err_est, converged).
    """
    sel = (lambda v: v) if top is None else top
    y = y0
    p = d[0] * y0
    if force_iters is not None and force_iters >= 0:
        for m in range(force_iters):
            y = matvec_shifted(y, m) - xi[m] * y
            p = p + d[m + 1] * y
        ny, np_ = np.linalg.norm(sel(y)), np.linalg.norm(sel(p))
        est = abs(d[force_iters]) * ny / np_ if np_ > 0 else 0.0
        return p, force_iters, est, True
    for m in range(max_iters):
        y = matvec_shifted(y, m) - xi[m] * y
        p = p + d[m + 1] * y
        ny, np_ = np.linalg.norm(sel(y)), np.linalg.norm(sel(p))
        if not (np.isfinite(ny) and np.isfinite(np_)):
            # a NaN, or terms that overflowed: the series has failed (without
            # this, inf <= inf would pass the test below as converged)
            return p, m + 1, float("inf"), False
        if m + 1 >= 2 and abs(d[m + 1]) * ny <= tol * np_:
            est = abs(d[m + 1]) * ny / np_ if np_ > 0 else 0.0
            return p, m + 1, est, True
    ny, np_ = np.linalg.norm(sel(y)), np.linalg.norm(sel(p))
    est = abs(d[max_iters]) * ny / np_ if np_ > 0 else float("inf")
    return p, max_iters, est, False


def leja_phi1(A, v, dt, alpha, tol=1e-10, force_iters=None, rho_max=200.0,
              max_iters=MAX_ITERS, adaptive=False):
    """out ~ phi_1(dt A) v by Leja interpolation of f(xi) = phi_1((c + gamma xi) h).

    Substeps (reading): with h = dt/K, w_0 = 0 and
    w_{k+1} = w_k + h phi_1(h A)(A w_k + v), w_K = dt phi_1(dt A) v, so
    out = w_K / dt (for K = 1 this is the single series itself).  The same
    recursion holds for unequal substeps (adaptive control).
    Returns (out, LejaStats).
    """
    if adaptive and not (force_iters is not None and force_iters >= 0):
        return _leja_phi1_adaptive(A, v, dt, alpha, tol, rho_max, max_iters)
    c, gamma = shift_scale(alpha)
    K = n_substeps(alpha, dt, rho_max)
    h = dt / K
    xi = leja_points(max_iters + 1)
    d = divided_differences(xi, phi1_scalar((c + gamma * xi) * h))
    mv = lambda y, m: (A @ y - c * y) / gamma
    st = LejaStats(substeps=K)
    v = np.asarray(v, dtype=np.float64)
    acc = np.zeros_like(v)
    w = np.zeros_like(v)
    for k in range(K):
        rhs = v if k == 0 else A @ w + v
        if k > 0:
            st.matvecs += 1
        q, it, est, ok = _newton_series(mv, rhs, d, xi, tol, force_iters, max_iters)
        st.iters += it
        st.matvecs += it
        st.err_est = max(st.err_est, est)
        st.converged &= ok
        acc = acc + q
        w = w + h * q
    return acc / K, st


def _leja_phi1_adaptive(A, v, dt, alpha, tol, rho_max, max_iters):
    c, gamma = shift_scale(alpha)
    xi = leja_points(max_iters + 1)
    mv = lambda y, m: (A @ y - c * y) / gamma
    v = np.asarray(v, dtype=np.float64)
    st = LejaStats()
    state = {"w": np.zeros_like(v), "rhs": v, "q": None, "n": 0}

    def attempt(h):
        if state["q"] is not None:            # commit the previous accepted attempt
            state["w"] = state["w"] + state["h"] * state["q"]
            state["rhs"] = A @ state["w"] + v
            st.matvecs += 1
            state["q"] = None
        d = divided_differences(xi, phi1_scalar((c + gamma * xi) * h))
        q, it, est, ok = _newton_series(mv, state["rhs"], d, xi, tol, None, max_iters)
        st.iters += it
        st.matvecs += it
        if ok:
            st.err_est = max(st.err_est, est)
            state["q"], state["h"] = q, h
            state["n"] += 1
        return ok, it

    K0 = n_substeps(alpha, dt, rho_max)
    sizes, rejected, ok, _ = adaptive_substeps(dt, K0, max_iters, attempt)
    st.substeps, st.rejected, st.sizes, st.converged = len(sizes), rejected, tuple(sizes), ok
    if not ok:
        return v.copy(), st
    if len(sizes) == 1:
        return state["q"], st
    w = state["w"] + state["h"] * state["q"]
    return w / dt, st


def leja_exp_augmented(A, x0, eta0, w1, w2, dt, alpha, tol=1e-10, force_iters=None,
                       rho_max=200.0, max_iters=MAX_ITERS, adaptive=False):
    """Top block of exp(dt Atilde) [x0; eta0] for Atilde = [[A, W], [0, J]],
    W = [w2, w1], J = [[0, 1], [0, 0]] (Section 2: the sum of phi_l terms of
    Eq. exp_quad_Gauss is evaluated as the exponential of an augmented matrix).

    With x0 = 0 and eta0 = (0, 1) the top block equals
    dt phi_1(dt A) w1 + dt^2 phi_2(dt A) w2.  Substeps apply exp(h Atilde) K
    times.  Norms in the stopping rule use the top (length-N) block.
    Returns (top, eta, LejaStats).
    """
    c, gamma = shift_scale(alpha)
    K = n_substeps(alpha, dt, rho_max)
    h = dt / K
    xi = leja_points(max_iters + 1)
    n = len(x0)

    def mv(yt, m):
        y, e1, e2 = yt[:n], yt[n], yt[n + 1]
        top = A @ y + w2 * e1 + w1 * e2
        out = np.empty_like(yt)
        out[:n] = top
        out[n] = e2
        out[n + 1] = 0.0
        return (out - c * yt) / gamma

    state = np.concatenate([np.asarray(x0, dtype=np.float64), np.asarray(eta0, dtype=np.float64)])
    top = lambda v: v[:n]
    if adaptive and not (force_iters is not None and force_iters >= 0):
        st = LejaStats()
        cur = {"state": state, "new": None}

        def attempt(hs):
            if cur["new"] is not None:          # commit the previous accepted attempt
                cur["state"], cur["new"] = cur["new"], None
            dd = divided_differences(xi, np.exp((c + gamma * xi) * hs))
            new, it, est, ok = _newton_series(mv, cur["state"], dd, xi, tol, None, max_iters,
                                              top=top)
            st.iters += it
            st.matvecs += it
            if ok:
                st.err_est = max(st.err_est, est)
                cur["new"] = new
            return ok, it

        sizes, rejected, ok, _ = adaptive_substeps(dt, K, max_iters, attempt)
        st.substeps, st.rejected, st.sizes, st.converged = len(sizes), rejected, tuple(sizes), ok
        final = cur["new"] if ok else state
        return final[:n], final[n:], st
    d = divided_differences(xi, np.exp((c + gamma * xi) * h))
    st = LejaStats(substeps=K)
    for k in range(K):
        state, it, est, ok = _newton_series(mv, state, d, xi, tol, force_iters, max_iters,
                                            top=lambda v: v[:n])
        st.iters += it
        st.matvecs += it
        st.err_est = max(st.err_est, est)
        st.converged &= ok
    return state[:n], state[n:], st
