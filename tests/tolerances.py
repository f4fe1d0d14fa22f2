"""Tolerances of the parity tests, derived from the arithmetic.

Filter application (eq. disc_filtercoeff). Write u^_n = u_n + e_n for the
computed leapfrog states. Each step adds a local rounding error d_n with
||d_n||_M <= c_loc * eps * ||u^_n||_M (the row dot product of <= 16 terms,
the scale by tau^2/m and the three-term update: c_loc ~ 16 * (tau^2 G + 3)
with tau^2 G <= 4 under the CFL bound, G the Gershgorin bound of M^-1 S).
The error obeys the same two-step recurrence, e_{n+1} = (2 - tau^2 M^-1 S) e_n
- e_{n-1} + d_n, so e_n = sum_j U_{n-1-j}(I - tau^2 M^-1 S / 2) d_j with the
Chebyshev polynomials U_k of the second kind, |U_k| <= k + 1 on the stable
spectrum; ||u_n||_M <= ||r||_M / cos(theta_max / 2) (the third-kind bound of
eq. scalartimestep). Summing with the weights gives the first-order bound

    ||C^ r - C r||_M <= (sum_n |alpha_n|) * c_loc * eps * L^2 / (2 cos(theta_max/2)) * ||r||_M,

i.e. about 130 * eps * L^2 after normalising by sum |alpha_n| ||r||_M. That
worst case assumes every rounding error has the same sign and the largest
size. The tests use the probabilistic form of the same analysis (Higham &
Mary, SIAM J. Sci. Comput. 2019: independent, zero-mean rounding errors
accumulate like a random walk, with the same bound up to a small constant
holding with overwhelming probability):
  * a row's local error is the sum of ~w + 3 independent roundings (w <= 16
    products and sums of the row, the scale and the three-term update) of
    terms whose sizes add up to at most (tau^2 G + 3) |u| <= 7 |u|; spread over
    ~18 roundings that is a standard deviation of ~7/sqrt(18) ~ 1.7 eps |u|,
    and c_loc = 4 also covers the partial sums carried through the row;
  * the weighted sum sum_n alpha_n e_n = sum_j G_j d_j, where
    G_j = sum_{n>j} alpha_n U_{n-1-j} is bounded by sum |alpha_n| / sin(theta)
    and sin(theta) >= tau omega_min / 2 keeps it within a factor ~ 2 on the
    meshes used here; L independent terms then add to
    ~ 2 c_loc eps sqrt(L) sum |alpha_n| ||r||_M.
FILTER_TOL_C = 32 = 2 * c_loc * (safety factor 4). The FP32 form has
eps = 2^-24 for values and state; its accumulator is compensated (two-sum and
two-product), so the sum adds no error of its own.

Eigenvalues: the targets are a relative 1e-10 (FP64 form) and 1e-6 (FP32 form)
against the exact (closed-form) spectrum.
"""
import numpy as np

EPS64 = float(np.finfo(np.float64).eps) / 2     # unit roundoff 2^-53
EPS32 = float(np.finfo(np.float32).eps) / 2     # 2^-24
FILTER_WORST_C = 130.0
FILTER_TOL_C = 32.0

EIG_REL = {"fp64": 1e-10, "fp32": 1e-6}


# Fourth-order stepper (stage v = u + A u / 12, then the step gathers A v): the stage's
# rounding, about 2 eps |u| (its row sum of terms adding up to ||A|| / 12 |u| <= |u|, and
# the final add), reaches u_{n+1} through A, ||A|| = tau^2 ||M^-1 S|| <= 0.81 * 12 ~ 10 at
# 0.9 of its CFL bound: c_loc grows from ~4 to ~4 + 10 * 2 = 24, six times the leapfrog's.
FILTER4_TOL_C = 6 * FILTER_TOL_C


def filter_tol_leapfrog4(L: int, precision: str) -> float:
    """filter_tol for the fourth-order modified-equation leapfrog."""
    eps = EPS64 if precision == "fp64" else EPS32
    return FILTER4_TOL_C * eps * (L + 1) ** 0.5


def filter_tol(L: int, precision: str) -> float:
    """Tolerance on ||C_gpu r - C_oracle r||_M / (sum_n |alpha_n| * ||r||_M)."""
    eps = EPS64 if precision == "fp64" else EPS32
    return FILTER_TOL_C * eps * (L + 1) ** 0.5


def filter_worst_bound(L: int, precision: str) -> float:
    """First-order worst-case bound (every rounding error aligned)."""
    eps = EPS64 if precision == "fp64" else EPS32
    return FILTER_WORST_C * eps * L * L


def filter_error(got: np.ndarray, ref: np.ndarray, r: np.ndarray, m: np.ndarray,
                 alpha: np.ndarray) -> float:
    """||got - ref||_M / (sum |alpha| ||r||_M) for one vector (or row-stacked vectors)."""
    got, ref, r = np.atleast_2d(got), np.atleast_2d(ref), np.atleast_2d(r)
    num = np.sqrt(np.sum((got - ref) ** 2 * m, axis=-1))
    den = np.abs(alpha).sum() * np.sqrt(np.sum(r ** 2 * m, axis=-1))
    return float(np.max(num / den))


def elementwise_bound(tol: float, r: np.ndarray, m: np.ndarray, alpha: np.ndarray) -> float:
    """Entry-wise bound implied by the M-norm bound: |e_i| <= ||e||_M / sqrt(min m)."""
    rm = np.sqrt(np.sum(np.atleast_2d(r) ** 2 * m, axis=-1)).max()
    return tol * np.abs(alpha).sum() * rm / np.sqrt(m.min())


def fp32_residual_floor(S, m: np.ndarray, omega_min: float) -> float:
    """Relative residual that Ritz pairs of the FP32 form cannot be expected to beat.

    The FP32 form stores the step values A = -tau^2 M^-1 S rounded once to FP32, a relative
    error of at most 2^-24 per entry, so its Krylov space belongs to the perturbed operator
    K~ = K + dK with |dK| <= 2^-24 |K| entrywise (K = M^-1 S). An eigenvector x of K~ has
    ||(K - theta) x||_inf <= 2^-24 G ||x||_inf, G = max_i sum_j |s_ij| / m_i (the Gershgorin
    bound of |K|); relative to theta >= omega_min^2 that is at most 2^-24 G / omega_min^2.
    Pairs near this level pass or fail an acceptance test by chance, so a count of accepted
    pairs is only compared well above it."""
    G = float(np.max(np.asarray(abs(S).sum(axis=1)).ravel() / m))
    return EPS32 * G / (omega_min * omega_min)
