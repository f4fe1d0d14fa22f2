"""Oracle: a plain, slow FP64 CPU restatement of the filtered time-domain
Krylov eigensolver of Nannen & Wess, "A Krylov Eigenvalue Solver Based on
Filtered Time Domain Solutions" (arXiv:2402.08515), Sec. 2.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU
baseline / reference arm of bench.py import this module. The CUDA library
never calls it, links it or shares code with it; the two meet only through
the seeded inputs of ``fe_inputs``.

Everything is float64 numpy; the sparse product S @ y is scipy's CSR matvec
(a library primitive) and the small symmetric eigenproblem is LAPACK through
numpy.linalg.eigh. Steps are taken in the paper's order and notation; where
the paper is silent or garbled the reading taken is stated in the docstring.

Readings used throughout (see the function docstrings):
  * index range: ``L`` time steps give the L+1 samples y_0..y_L, weighted by
    alpha_n = tau * alpha(n tau), n = 0..L, so the last sample is at t = T = L tau
    (eq. disc_filtercoeff sums l = 0..L-1 with L-1 steps; the closed interval
    (0, T] of eq. weightf is covered by taking L steps and L+1 terms);
  * inner product: the M-inner product (x, y)_M = x^T M y with two full
    classical Gram-Schmidt passes (Algorithm 2.5 uses the Euclidean product
    and one modified pass); the projected problem eq. projevp then becomes a
    standard symmetric eigenproblem because B^T M B = I;
  * breakdown: stop when the M-norm after orthogonalisation is below 1e-10
    times the M-norm before it (Algorithm 2.5 tests for an exact zero);
  * Krylov dimension kmax = number of basis vectors b_0..b_{kmax-1}, which
    takes kmax-1 filter applications;
  * residual: rel_res = ||S x - theta M x||_2 / (theta ||M x||_2) with
    x = B y, ||x||_M = 1; the absolute residual of eq. res is also returned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "weight", "alpha_table", "q_values", "beta_tilde", "filter_apply",
    "filter_apply_multi", "power_iteration", "m_inner", "m_norm",
    "orthonormalize_cgs2", "rayleigh_ritz", "ritz_residuals", "krylov_solve",
    "block_krylov_solve", "multi_interval_krylov_solve", "subspace_iteration",
    "refine_subspace", "refine_selection", "gaussian_weight", "alpha_table_gaussian", "triangle_weight",
    "alpha_table_triangle", "q_values_leapfrog4", "beta_tilde_leapfrog4",
    "filter_apply_leapfrog4",
    "KrylovResult", "BREAKDOWN_RATIO",
]

BREAKDOWN_RATIO = 1e-10


# --------------------------------------------------------------------------
# weight function and weight table: eq. (weightf), eq. (disc_filtercoeff)
# --------------------------------------------------------------------------

def weight(t, omega_min: float, omega_max: float, T: float):
    """alpha(t) of eq. (weightf).

    alpha(0) = 2 (omega_max - omega_min) / pi; for 0 < t <= T
    alpha(t) = 4/(pi t) sin(t (omega_max - omega_min)/2) cos(t (omega_max + omega_min)/2);
    alpha(t) = 0 for t > T.
    """
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    zero = t == 0.0
    inside = (t > 0.0) & (t <= T)
    out[zero] = 2.0 * (omega_max - omega_min) / math.pi
    ti = t[inside]
    out[inside] = (4.0 / (math.pi * ti) * np.sin(0.5 * ti * (omega_max - omega_min))
                   * np.cos(0.5 * ti * (omega_max + omega_min)))
    return out


def alpha_table(omega_min: float, omega_max: float, tau: float, L: int) -> np.ndarray:
    """Rectangle-rule weights alpha_n = tau * alpha(n tau), n = 0..L, T = L tau
    (eq. disc_filtercoeff with the L-steps / L+1-terms reading)."""
    T = L * tau
    n = np.arange(L + 1, dtype=np.float64)
    return tau * weight(n * tau, omega_min, omega_max, T)


def gaussian_weight(t, center: float, sigma: float):
    """Weight of a Gaussian pass band (Sec. 4, "Weight function": a Gaussian peak in
    place of the indicator). With beta_alpha(s) = int_0^inf alpha(t) cos(ts) dt
    (eq. filterfunc) and its inverse alpha(t) = (2/pi) int_0^inf beta(s) cos(ts) ds
    (the transform eq. filterf applies to the indicator), the even band
    beta(s) = exp(-(s-c)^2 / (2 sigma^2)) + exp(-(s+c)^2 / (2 sigma^2)) gives
    alpha(t) = 2 sigma sqrt(2/pi) exp(-sigma^2 t^2 / 2) cos(c t)."""
    t = np.asarray(t, dtype=np.float64)
    return 2.0 * sigma * math.sqrt(2.0 / math.pi) * np.exp(-0.5 * sigma * sigma * t * t) * np.cos(center * t)


def alpha_table_gaussian(center: float, sigma: float, tau: float, L: int) -> np.ndarray:
    """Rectangle-rule weights tau * alpha(n tau), n = 0..L, of the Gaussian band."""
    return tau * gaussian_weight(np.arange(L + 1, dtype=np.float64) * tau, center, sigma)


def triangle_weight(t, center: float, half_width: float):
    """Weight of a triangular (hat) pass band (Sec. 4, "Weight function"). For the even
    band beta(s) = hat(s - c) + hat(s + c), hat(u) = max(0, 1 - |u| / h), the inverse
    transform alpha(t) = (2/pi) int_0^inf beta(s) cos(ts) ds is (1/pi) times the integral
    over the whole line, i.e. (2/pi) cos(c t) int hat(u) cos(t u) du, and the integral of
    the hat against cos(t u) is h (sin(t h / 2) / (t h / 2))^2."""
    t = np.asarray(t, dtype=np.float64)
    x = 0.5 * t * half_width
    sinc = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    return 2.0 * half_width / math.pi * np.cos(center * t) * sinc * sinc


def alpha_table_triangle(center: float, half_width: float, tau: float, L: int) -> np.ndarray:
    """Rectangle-rule weights tau * alpha(n tau), n = 0..L, of the triangular band."""
    return tau * triangle_weight(np.arange(L + 1, dtype=np.float64) * tau, center, half_width)


# --------------------------------------------------------------------------
# discrete filter: eq. (scalartimestep), eq. (fullydiscfilter)
# --------------------------------------------------------------------------

def q_values(omega, tau: float, L: int) -> np.ndarray:
    """q_l(omega), l = 0..L, of the scalar recurrence eq. (scalartimestep):
    q_{-1} = q_0 = 1, q_{l+1} = (2 - tau^2 omega^2) q_l - q_{l-1}.
    Returns shape (L+1, len(omega))."""
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    q = np.empty((L + 1, omega.size))
    q_prev = np.ones_like(omega)
    q_cur = np.ones_like(omega)
    q[0] = q_cur
    for l in range(L):
        q_next = (2.0 - tau * tau * omega * omega) * q_cur - q_prev
        q[l + 1] = q_next
        q_prev, q_cur = q_cur, q_next
    return q


def beta_tilde(omega, alpha: np.ndarray, tau: float) -> np.ndarray:
    """Fully discrete filter of eq. (fullydiscfilter):
    beta~(omega) = sum_{n=0..L} alpha_n q_n(omega), alpha_n = tau alpha(n tau)."""
    L = len(alpha) - 1
    return alpha @ q_values(omega, tau, L)


# --------------------------------------------------------------------------
# filter application: eq. (2stepmethod) + eq. (disc_filtercoeff)
# --------------------------------------------------------------------------

def filter_apply(S, m: np.ndarray, r: np.ndarray, tau: float,
                 alpha: np.ndarray) -> np.ndarray:
    """C r = sum_{n=0..L} alpha_n y_n(r) (eq. disc_filtercoeff).

    y_{-1} = y_0 = r and y_{l+1} = -tau^2 M^{-1} S y_l + 2 y_l - y_{l-1}
    (eq. 2stepmethod), M = diag(m); the inner loop of Algorithm 2.5."""
    L = len(alpha) - 1
    y_prev = np.array(r, dtype=np.float64)
    y = np.array(r, dtype=np.float64)
    acc = alpha[0] * y
    for l in range(L):
        y_next = -tau * tau * (S @ y) / m + 2.0 * y - y_prev
        acc = acc + alpha[l + 1] * y_next
        y_prev, y = y, y_next
    return acc


# --------------------------------------------------------------------------
# another time stepper (Remark 2.4, Sec. 4 "Time-stepping"): the fourth-order
# modified-equation leapfrog. Like eq. (2stepmethod) it is diagonalised by the
# eigenvectors, so Lemma 2.3 holds with its own scalar recurrence.
# --------------------------------------------------------------------------

def q_values_leapfrog4(omega, tau: float, L: int) -> np.ndarray:
    """q_l(omega), l = 0..L, of the fourth-order scheme on one eigenvector:
    q_{-1} = q_0 = 1, q_{l+1} = (2 - x + x^2 / 12) q_l - q_{l-1}, x = tau^2 omega^2.
    Returns shape (L+1, len(omega))."""
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    x = tau * tau * omega * omega
    a = 2.0 - x + x * x / 12.0
    q = np.empty((L + 1, omega.size))
    q_prev = np.ones_like(omega)
    q_cur = np.ones_like(omega)
    q[0] = q_cur
    for l in range(L):
        q_next = a * q_cur - q_prev
        q[l + 1] = q_next
        q_prev, q_cur = q_cur, q_next
    return q


def beta_tilde_leapfrog4(omega, alpha: np.ndarray, tau: float) -> np.ndarray:
    """The factor the fourth-order filter applies to an eigenvector of frequency
    omega: sum_{n=0..L} alpha_n q_n(omega) with q_values_leapfrog4."""
    L = len(alpha) - 1
    return alpha @ q_values_leapfrog4(omega, tau, L)


def filter_apply_leapfrog4(S, m: np.ndarray, r: np.ndarray, tau: float,
                           alpha: np.ndarray) -> np.ndarray:
    """sum_{n=0..L} alpha_n y_n(r) for the fourth-order modified-equation leapfrog
    y_{l+1} = 2 y_l - y_{l-1} - tau^2 K y_l + (tau^4 / 12) K^2 y_l, K = M^{-1} S,
    from y_{-1} = y_0 = r (the start of eq. 12). Stable for tau omega_max <= 2 sqrt(3)."""
    L = len(alpha) - 1
    y_prev = np.array(r, dtype=np.float64)
    y = np.array(r, dtype=np.float64)
    acc = alpha[0] * y
    for l in range(L):
        Ky = (S @ y) / m
        KKy = (S @ Ky) / m
        y_next = 2.0 * y - y_prev - tau * tau * Ky + tau ** 4 / 12.0 * KKy
        acc = acc + alpha[l + 1] * y_next
        y_prev, y = y, y_next
    return acc


def filter_apply_multi(S, m: np.ndarray, R: np.ndarray, tau: float,
                       alphas: np.ndarray) -> np.ndarray:
    """Several weight tables on one trajectory per start vector.

    R: (b, n) start vectors; alphas: (F, L+1) weight tables sharing tau and L.
    Returns (F, b, n) with out[f, j] = sum_n alphas[f, n] y_n(R[j])."""
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    alphas = np.atleast_2d(np.asarray(alphas, dtype=np.float64))
    F, Lp1 = alphas.shape
    out = np.empty((F, R.shape[0], R.shape[1]))
    for j in range(R.shape[0]):
        y_prev = R[j].copy()
        y = R[j].copy()
        acc = [alphas[f, 0] * y for f in range(F)]
        for l in range(Lp1 - 1):
            y_next = -tau * tau * (S @ y) / m + 2.0 * y - y_prev
            for f in range(F):
                acc[f] = acc[f] + alphas[f, l + 1] * y_next
            y_prev, y = y, y_next
        for f in range(F):
            out[f, j] = acc[f]
    return out


# --------------------------------------------------------------------------
# power iteration for omega_max(S, M) (Sec. 3.1: the stable time step is
# "determined using a power iteration")
# --------------------------------------------------------------------------

def power_iteration(S, m: np.ndarray, v0: np.ndarray, iters: int) -> float:
    """Largest eigenfrequency of the pencil by power iteration on M^{-1} S.

    v <- M^{-1} S v / ||M^{-1} S v||_2, ``iters`` times from v0/||v0||_2; the
    estimate is sqrt of the Rayleigh quotient (v^T S v)/(v^T M v)."""
    v = np.array(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    for _ in range(iters):
        w = (S @ v) / m
        v = w / np.linalg.norm(w)
    theta = (v @ (S @ v)) / (v @ (m * v))
    return math.sqrt(theta)


# --------------------------------------------------------------------------
# Gram-Schmidt in the M-inner product (Algorithm 2.5, orthogonalisation loop)
# --------------------------------------------------------------------------

def m_inner(x: np.ndarray, y: np.ndarray, m: np.ndarray) -> float:
    return float(np.sum(x * m * y))


def m_norm(x: np.ndarray, m: np.ndarray) -> float:
    return math.sqrt(m_inner(x, x, m))


def orthonormalize_cgs2(B: np.ndarray, w: np.ndarray, m: np.ndarray):
    """Two classical Gram-Schmidt passes of w against the columns of B in the
    M-inner product, then M-normalisation.

    B: (k, n) with M-orthonormal rows. Returns (b, norm_before, norm_after);
    b is None on breakdown (norm_after < BREAKDOWN_RATIO * norm_before)."""
    w = np.array(w, dtype=np.float64)
    norm_before = m_norm(w, m)
    for _ in range(2):
        if B.shape[0]:
            h = B @ (m * w)           # h_j = (w, b_j)_M
            w = w - h @ B             # w -= sum_j h_j b_j
    norm_after = m_norm(w, m)
    if not norm_after > BREAKDOWN_RATIO * norm_before:
        return None, norm_before, norm_after
    return w / norm_after, norm_before, norm_after


# --------------------------------------------------------------------------
# Rayleigh-Ritz (eq. projevp) and residuals (eq. res)
# --------------------------------------------------------------------------

def rayleigh_ritz(S, B: np.ndarray):
    """Eigenpairs of B^T S B y = theta B^T M B y with B^T M B = I.

    B: (k, n), rows M-orthonormal. Returns ascending theta (k,) and Y (k, k)
    with columns y_j. Negative theta from rounding is clamped to 0 (S PSD)."""
    SB = np.stack([S @ b for b in B]) if B.shape[0] else np.zeros_like(B)
    H = B @ SB.T                      # H[i, j] = b_i^T S b_j
    H = 0.5 * (H + H.T)
    theta, Y = np.linalg.eigh(H)
    return np.maximum(theta, 0.0), Y


def ritz_residuals(S, m: np.ndarray, B: np.ndarray, theta: np.ndarray,
                   Y: np.ndarray):
    """For each Ritz pair: x = B^T y (||x||_M = 1), the absolute residual
    ||(S - theta M) x||_2 of eq. (res) and the relative one
    ||S x - theta M x||_2 / (theta ||M x||_2). Returns (X (p, n), abs, rel)."""
    X = Y.T @ B
    abs_res = np.empty(len(theta))
    rel_res = np.empty(len(theta))
    for j, (th, x) in enumerate(zip(theta, X)):
        r = S @ x - th * (m * x)
        abs_res[j] = np.linalg.norm(r)
        denom = th * np.linalg.norm(m * x)
        rel_res[j] = abs_res[j] / denom if denom > 0 else math.inf
    return X, abs_res, rel_res


# --------------------------------------------------------------------------
# the Krylov eigensolver (Algorithm 2.5 + eq. projevp + eq. res)
# --------------------------------------------------------------------------

@dataclass
class KrylovResult:
    omega2: np.ndarray            # accepted theta, ascending
    omega: np.ndarray
    rel_res: np.ndarray
    abs_res: np.ndarray
    vectors: np.ndarray           # (p, n)
    k_used: int                   # basis size reached
    time_steps: int               # leapfrog steps taken
    breakdown: bool
    ritz_theta: np.ndarray        # every Ritz value of the last projection
    ritz_rel_res: np.ndarray      # rel. residual of the in-interval ones (nan elsewhere)
    basis: np.ndarray             # (k_used, n)
    history: list = field(default_factory=list)
    interval: np.ndarray = None   # index of the interval each accepted pair lies in


def krylov_solve(S, m: np.ndarray, r0: np.ndarray, omega_min: float,
                 omega_max: float, tau: float, L: int, kmax: int, tol: float,
                 check_every: int = 5, keep_basis: bool = True) -> KrylovResult:
    """Krylov space of C from r0 (Algorithm 2.5), projected problem
    (eq. projevp) and residual acceptance (eq. res).

    b_0 = r0/||r0||_M; for k = 0.. : w = C b_k, CGS2 in the M-inner product,
    stop on breakdown, b_{k+1} = w/||w||_M, until kmax basis vectors exist.
    Every ``check_every`` new vectors and at the end the projected problem is
    solved; pairs with omega = sqrt(theta) in [omega_min, omega_max] and
    rel_res <= tol are accepted (the last projection is returned)."""
    alpha = alpha_table(omega_min, omega_max, tau, L)
    n = len(m)
    B = np.zeros((kmax, n))
    B[0] = r0 / m_norm(r0, m)
    k = 1
    steps = 0
    breakdown = False
    history = []

    def project(k):
        theta, Y = rayleigh_ritz(S, B[:k])
        omega = np.sqrt(theta)
        inside = (omega >= omega_min) & (omega <= omega_max)
        rel_all = np.full(k, np.nan)
        X, a, r = ritz_residuals(S, m, B[:k], theta[inside], Y[:, inside])
        rel_all[inside] = r
        acc = r <= tol
        history.append(dict(k=k, n_inside=int(inside.sum()), n_acc=int(acc.sum())))
        return theta, rel_all, theta[inside][acc], r[acc], a[acc], X[acc]

    while k < kmax:
        w = filter_apply(S, m, B[k - 1], tau, alpha)
        steps += L
        b, nb, na = orthonormalize_cgs2(B[:k], w, m)
        if b is None:
            breakdown = True
            break
        B[k] = b
        k += 1
        if k % check_every == 0 and k < kmax:
            project(k)
    theta, rel_all, th_acc, rel_acc, abs_acc, X_acc = project(k)
    return KrylovResult(omega2=th_acc, omega=np.sqrt(th_acc), rel_res=rel_acc,
                        abs_res=abs_acc, vectors=X_acc, k_used=k,
                        time_steps=steps, breakdown=breakdown, ritz_theta=theta,
                        ritz_rel_res=rel_all,
                        basis=B[:k] if keep_basis else None, history=history)


def block_krylov_solve(S, m: np.ndarray, R0: np.ndarray, omega_min: float,
                       omega_max: float, tau: float, L: int, kmax: int, tol: float,
                       check_every: int = 5, keep_basis: bool = True) -> KrylovResult:
    """Block version of the Krylov space (Sec. 4, eigenvalue solver): start from b
    M-orthonormalised random vectors and orthonormalise every filtered block.

    R0: (b, n). The b start vectors are orthonormalised in order (CGS2, dependent
    ones dropped). Each block step filters the b newest basis vectors, one after the
    other orthogonalises each filtered vector into the basis and appends it unless it
    is dependent, stopping at kmax vectors; a step that appends nothing is a
    breakdown. The projected problem and the acceptance are those of krylov_solve,
    solved whenever the basis size passes a multiple of check_every and at the end."""
    R0 = np.atleast_2d(np.asarray(R0, dtype=np.float64))
    b = R0.shape[0]
    alpha = alpha_table(omega_min, omega_max, tau, L)
    n = len(m)
    B = np.zeros((kmax, n))
    k = 0
    for r in R0:
        if k >= kmax:
            break
        v, nb, na = orthonormalize_cgs2(B[:k], r, m)
        if v is not None:
            B[k] = v
            k += 1
    steps = 0
    breakdown = k == 0
    history = []
    next_check = check_every

    def project(kk):
        theta, Y = rayleigh_ritz(S, B[:kk])
        omega = np.sqrt(theta)
        inside = (omega >= omega_min) & (omega <= omega_max)
        rel_all = np.full(kk, np.nan)
        X, a, r = ritz_residuals(S, m, B[:kk], theta[inside], Y[:, inside])
        rel_all[inside] = r
        acc = r <= tol
        history.append(dict(k=kk, n_inside=int(inside.sum()), n_acc=int(acc.sum())))
        return theta, rel_all, theta[inside][acc], r[acc], a[acc], X[acc]

    kproj = -1
    while not breakdown and k < kmax:
        newest = [B[j] if j >= 0 else np.zeros(n) for j in range(k - b, k)]
        W = [filter_apply(S, m, v, tau, alpha) for v in newest]
        steps += L
        added = 0
        for w in W:
            if k >= kmax:
                break
            v, nb, na = orthonormalize_cgs2(B[:k], w, m)
            if v is None:
                continue
            B[k] = v
            k += 1
            added += 1
        if added == 0:
            breakdown = True
            break
        if k >= next_check and k < kmax:
            while next_check <= k:
                next_check += check_every
            project(k)
            kproj = k
    theta, rel_all, th_acc, rel_acc, abs_acc, X_acc = project(k)
    return KrylovResult(omega2=th_acc, omega=np.sqrt(th_acc), rel_res=rel_acc,
                        abs_res=abs_acc, vectors=X_acc, k_used=k,
                        time_steps=steps, breakdown=breakdown, ritz_theta=theta,
                        ritz_rel_res=rel_all,
                        basis=B[:k] if keep_basis else None, history=history)


def multi_interval_krylov_solve(S, m: np.ndarray, R0: np.ndarray, intervals, tau: float,
                                L: int, kmax: int, tol: float, check_every: int = 5,
                                refine_sweeps: int = 0, refine_extra: int = 0) -> KrylovResult:
    """F intervals searched at once by F independent block Krylov processes.

    R0: (b, n) with b a multiple of F = len(intervals); g = b / F. Process f is the
    block solver of Sec. 4 (block_krylov_solve) on interval f from the start vectors
    R0[f g : (f + 1) g], with its own basis of up to kmax vectors; the processes only
    share the time stepping (column j of the b-column trajectory belongs to process
    j // g), which does not change what any of them computes. With refine_sweeps > 0,
    each process's in-interval Ritz vectors (and the refine_extra nearest outside
    its interval) then go through refine_subspace on its interval. The accepted pairs of all processes are merged in ascending theta with
    the index of the interval that found each (a pair in two overlapping intervals
    is reported by both); k_used adds up over the processes, time_steps is the length
    of the shared trajectory (the most steps any process took), and the Ritz values
    of the last projections are listed process after process."""
    R0 = np.atleast_2d(np.asarray(R0, dtype=np.float64))
    b = R0.shape[0]
    F = len(intervals)
    if F < 1 or b % F:
        raise ValueError("the block width must be a multiple of the number of intervals")
    g = b // F
    parts = []
    for f, (lo, hi) in enumerate(intervals):
        r = block_krylov_solve(S, m, R0[f * g:(f + 1) * g], lo, hi, tau, L, kmax, tol,
                               check_every, keep_basis=refine_sweeps > 0)
        if refine_sweeps > 0:
            theta_r, Y = rayleigh_ritz(S, r.basis)
            X = (Y.T @ r.basis)[refine_selection(theta_r, lo, hi, refine_extra)]
            if len(X):
                th, rel, Xa, thi, reli = refine_subspace(S, m, X, lo, hi, tau, L, tol,
                                                         refine_sweeps, refine_extra)
                X_acc, a_acc = Xa, np.array([np.linalg.norm(S @ x - t * (m * x))
                                             for t, x in zip(th, Xa)])
                r = KrylovResult(omega2=th, omega=np.sqrt(th), rel_res=rel, abs_res=a_acc,
                                 vectors=X_acc, k_used=r.k_used, time_steps=r.time_steps,
                                 breakdown=r.breakdown, ritz_theta=r.ritz_theta,
                                 ritz_rel_res=r.ritz_rel_res, basis=None, history=r.history)
        parts.append(r)
    theta = np.concatenate([r.omega2 for r in parts])
    label = np.concatenate([np.full(len(r.omega2), f, dtype=np.int64) for f, r in enumerate(parts)])
    order = np.argsort(theta, kind="stable")
    n = len(m)
    return KrylovResult(
        omega2=theta[order], omega=np.sqrt(theta[order]),
        rel_res=np.concatenate([r.rel_res for r in parts])[order],
        abs_res=np.concatenate([r.abs_res for r in parts])[order],
        vectors=np.concatenate([np.reshape(r.vectors, (-1, n)) for r in parts])[order],
        k_used=sum(r.k_used for r in parts), time_steps=max(r.time_steps for r in parts),
        breakdown=any(r.breakdown for r in parts),
        ritz_theta=np.concatenate([r.ritz_theta for r in parts]),
        ritz_rel_res=np.concatenate([r.ritz_rel_res for r in parts]),
        basis=None, history=[r.history for r in parts], interval=label[order])


def refine_selection(theta: np.ndarray, omega_min: float, omega_max: float, extra: int = 0) -> np.ndarray:
    """Indices (ascending) of the Ritz values whose vectors a refinement sweep filters:
    every one with omega = sqrt(theta) in [omega_min, omega_max], and the `extra` nearest
    outside it (distance in omega to the interval, ties to the lower index), a buffer
    like the one FEAST keeps beyond the wanted eigenvalues."""
    omega = np.sqrt(np.maximum(np.asarray(theta, dtype=np.float64), 0.0))
    inside = (omega >= omega_min) & (omega <= omega_max)
    out = np.flatnonzero(~inside)
    dist = np.where(omega[out] < omega_min, omega_min - omega[out], omega[out] - omega_max)
    keep = out[np.argsort(dist, kind="stable")[:max(extra, 0)]]
    return np.sort(np.concatenate([np.flatnonzero(inside), keep]))


def refine_subspace(S, m: np.ndarray, X: np.ndarray, omega_min: float, omega_max: float,
                    tau: float, L: int, tol: float, sweeps: int = 1, extra: int = 0):
    """Filtered subspace iteration on the rows of X (the fixed-dimension, FEAST-like
    use of the filter mentioned in Sec. 4): each sweep filters every vector (X <- C X),
    M-orthonormalises the result (CGS2, dependent vectors dropped), solves the
    projected problem (eq. projevp) and keeps the Ritz vectors with omega in the
    interval, and the `extra` nearest outside it (refine_selection), for the next
    sweep. Returns (theta_acc, rel_acc, X_acc, theta_inside, rel_inside) of the last
    sweep, acceptance rel_res <= tol."""
    alpha = alpha_table(omega_min, omega_max, tau, L)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    th_in = rel_in = np.zeros(0)
    th_acc = rel_acc = np.zeros(0)
    X_acc = np.zeros((0, X.shape[1]))
    for _ in range(sweeps):
        B = np.zeros((0, X.shape[1]))
        for x in X:
            v, nb, na = orthonormalize_cgs2(B, filter_apply(S, m, x, tau, alpha), m)
            if v is not None:
                B = np.vstack([B, v])
        theta, Y = rayleigh_ritz(S, B)
        omega = np.sqrt(theta)
        inside = (omega >= omega_min) & (omega <= omega_max)
        Xi, a, r = ritz_residuals(S, m, B, theta[inside], Y[:, inside])
        th_in, rel_in = theta[inside], r
        acc = r <= tol
        th_acc, rel_acc, X_acc = th_in[acc], r[acc], Xi[acc]
        X = (Y.T @ B)[refine_selection(theta, omega_min, omega_max, extra)]
    return th_acc, rel_acc, X_acc, th_in, rel_in


def subspace_iteration(S, m: np.ndarray, X0: np.ndarray, omega_min: float, omega_max: float,
                       tau: float, L: int, tol: float, sweeps: int):
    """The fixed-dimension alternative of Sec. 4 (FEAST-like filtered subspace
    iteration): from the p rows of X0, each sweep filters every vector (X <- C X),
    M-orthonormalises them in order (CGS2, dependent vectors dropped), solves the
    projected problem (eq. projevp) and takes all of its Ritz vectors, ascending, as the
    next X, so the subspace keeps its dimension. The pairs of the last sweep with omega
    in the interval and rel_res <= tol are accepted. Returns (theta_acc, rel_acc, X_acc,
    theta_all, rel_inside) where rel_inside is nan outside the interval."""
    alpha = alpha_table(omega_min, omega_max, tau, L)
    X = np.atleast_2d(np.asarray(X0, dtype=np.float64))
    theta = np.zeros(0)
    rel_all = np.zeros(0)
    th_acc = rel_acc = np.zeros(0)
    X_acc = np.zeros((0, X.shape[1]))
    for _ in range(sweeps):
        B = np.zeros((0, X.shape[1]))
        for x in X:
            v, nb, na = orthonormalize_cgs2(B, filter_apply(S, m, x, tau, alpha), m)
            if v is not None:
                B = np.vstack([B, v])
        theta, Y = rayleigh_ritz(S, B)
        omega = np.sqrt(theta)
        inside = (omega >= omega_min) & (omega <= omega_max)
        Xi, a, r = ritz_residuals(S, m, B, theta[inside], Y[:, inside])
        rel_all = np.full(len(theta), np.nan)
        rel_all[inside] = r
        acc = r <= tol
        th_acc, rel_acc, X_acc = theta[inside][acc], r[acc], Xi[acc]
        X = Y.T @ B
    return th_acc, rel_acc, X_acc, theta, rel_all
