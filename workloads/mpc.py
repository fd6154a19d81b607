"""Seeded synthetic MPC workloads that feed both the solver and the oracle.

This module only *builds* quadratic programs; it contains none of the solver's
arithmetic (no ADMM step, no layer weights, no residual or penalty rule).
Every problem is a condensed, LQR-preconditioned linear MPC problem as in the
paper's "Dense Model-Predictive Control" section (Sec. IV; the direct form is
Eq. mpc_def of Sec. II-C):

    x_{k+1} = A x_k + B u_k,  u_k = -K x_k + du_k,  Abar = A - B K,
    y = S ytilde + M x0,  Hbar = S^T H S,  gbar = S^T H M x0,
    Gbar = G S,  cbar = c - G M x0,  dbar = d - G M x0.

The decision vector is ytilde = [du_0; ...; du_{N-1}] (n = N*nu).  The
constraints are the control limits |u_k| <= umax (m = N*nu rows), plus, for
the humanoid-sized workload, extra dense inequalities on ytilde.  A problem is
returned in *parametric* form so that a new initial state only changes
(q, l, u):

    q = F x0,   l = l0 - E x0,   u = u0 - E x0.

All randomness comes from ``numpy.random.default_rng(SeedSequence([a, b]))``
so that each (workload id, sub id) pair names one reproducible stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(workload_id: int, sub_id: int = 0) -> np.random.Generator:
    """Counter-free seeded stream for one (workload, sub-draw) pair."""
    return np.random.default_rng(np.random.SeedSequence([int(workload_id), int(sub_id)]))


@dataclass
class ParametricQP:
    """min 1/2 x^T P x + q^T x  s.t.  l <= A x <= u, with (q,l,u) affine in x0."""

    P: np.ndarray          # (n, n) symmetric positive definite
    A: np.ndarray          # (m, n) constraint matrix
    F: np.ndarray          # (n, nx): q = F x0
    E: np.ndarray          # (m, nx): l = l0 - E x0, u = u0 - E x0
    l0: np.ndarray         # (m,) may hold -inf
    u0: np.ndarray         # (m,) may hold +inf
    Ad: np.ndarray         # (nx, nx) plant dynamics
    Bd: np.ndarray         # (nx, nu) plant input matrix
    K: np.ndarray          # (nu, nx) LQR gain used as preconditioner
    N: int                 # horizon
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.P.shape[0]

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def nx(self) -> int:
        return self.Ad.shape[0]

    @property
    def nu(self) -> int:
        return self.Bd.shape[1]

    def instance(self, x0: np.ndarray):
        """(q, l, u) of the QP for initial state x0 (one column or a batch of rows)."""
        x0 = np.asarray(x0, dtype=np.float64)
        if x0.ndim == 1:
            q = self.F @ x0
            s = self.E @ x0
            return q, self.l0 - s, self.u0 - s
        q = x0 @ self.F.T
        s = x0 @ self.E.T
        return q, self.l0[None, :] - s, self.u0[None, :] - s

    def first_control(self, x0: np.ndarray, ytilde: np.ndarray) -> np.ndarray:
        """u_0 = -K x0 + du_0 applied to the plant in closed loop."""
        return -self.K @ x0 + ytilde[: self.nu]


# ---------------------------------------------------------------------------
# plant generators
# ---------------------------------------------------------------------------

def random_dynamics(rng: np.random.Generator, nx: int, nu: int, spectral_radius: float = 1.05):
    """A = I + 0.1 N(0,1), rescaled to the given spectral radius; B ~ N(0,1)."""
    A = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx))
    A *= spectral_radius / np.max(np.abs(np.linalg.eigvals(A)))
    B = rng.standard_normal((nx, nu))
    return A, B


def block_dynamics(rng: np.random.Generator, nx: int, nu: int, block: int = 10,
                   spectral_radius: float = 1.0):
    """Block-diagonal A; each block I + 0.1 N(0,1) rescaled to the spectral radius."""
    A = np.zeros((nx, nx))
    for s in range(0, nx, block):
        e = min(s + block, nx)
        blk = np.eye(e - s) + 0.1 * rng.standard_normal((e - s, e - s))
        blk *= spectral_radius / np.max(np.abs(np.linalg.eigvals(blk)))
        A[s:e, s:e] = blk
    B = rng.standard_normal((nx, nu))
    return A, B


def lqr_gain(A: np.ndarray, B: np.ndarray, Q: np.ndarray, R: np.ndarray,
             tol: float = 1e-13, max_iter: int = 200000) -> np.ndarray:
    """Infinite-horizon discrete LQR gain by fixed-point Riccati iteration.

    X <- Q + A^T X A - A^T X B (R + B^T X B)^{-1} B^T X A, K = (R + B^T X B)^{-1} B^T X A.
    """
    X = Q.copy()
    for _ in range(max_iter):
        BtX = B.T @ X
        K = np.linalg.solve(R + BtX @ B, BtX @ A)
        Xn = Q + A.T @ X @ (A - B @ K)
        Xn = 0.5 * (Xn + Xn.T)
        if np.max(np.abs(Xn - X)) <= tol * max(1.0, np.max(np.abs(Xn))):
            X = Xn
            break
        X = Xn
    BtX = B.T @ X
    return np.linalg.solve(R + BtX @ B, BtX @ A)


def condensed_mpc(A: np.ndarray, B: np.ndarray, Q: np.ndarray, R: np.ndarray, QN: np.ndarray,
                  N: int, umax: float, precondition: bool = True):
    """Condensed (optionally LQR-preconditioned) MPC with box limits on u_k.

    Returns (P, Acon, F, E, l0, u0, K) for the decision vector du_0..du_{N-1}.
    """
    nx, nu = B.shape
    n = N * nu
    K = lqr_gain(A, B, Q, R) if precondition else np.zeros((nu, nx))
    Abar = A - B @ K
    # S_x[k] maps ytilde to x_{k+1} (k = 0..N-1); M_x[k] = Abar^{k+1}
    Sx = np.zeros((N, nx, n))
    Mx = np.zeros((N, nx, nx))
    Su = np.zeros((N, nu, n))
    Mu = np.zeros((N, nu, nx))
    xs_S = np.zeros((nx, n))          # x_0 part from ytilde is zero
    xs_M = np.eye(nx)
    for k in range(N):
        # u_k = -K x_k + du_k
        Su[k] = -K @ xs_S
        Su[k][:, k * nu:(k + 1) * nu] += np.eye(nu)
        Mu[k] = -K @ xs_M
        # x_{k+1} = Abar x_k + B du_k
        xs_S = Abar @ xs_S
        xs_S[:, k * nu:(k + 1) * nu] += B
        xs_M = Abar @ xs_M
        Sx[k] = xs_S
        Mx[k] = xs_M
    P = np.zeros((n, n))
    F = np.zeros((n, nx))
    for k in range(N):
        Wx = QN if k == N - 1 else Q
        P += Su[k].T @ R @ Su[k] + Sx[k].T @ Wx @ Sx[k]
        F += Su[k].T @ R @ Mu[k] + Sx[k].T @ Wx @ Mx[k]
    P = 0.5 * (P + P.T)
    Acon = Su.reshape(N * nu, n)
    E = Mu.reshape(N * nu, nx)
    l0 = -umax * np.ones(N * nu)
    u0 = umax * np.ones(N * nu)
    return P, Acon, F, E, l0, u0, K


def mpc_problem(nx: int, nu: int, N: int, umax: float, workload_id: int, *,
                dynamics: str = "random", spectral_radius: float = 1.05,
                extra_ineq: int = 0, name: str = "") -> ParametricQP:
    """One seeded parametric MPC QP (Q = I, R = 0.1 I, Q_N = Q)."""
    rng = rng_for(workload_id, 0)
    if dynamics == "random":
        Ad, Bd = random_dynamics(rng, nx, nu, spectral_radius)
    elif dynamics == "block":
        Ad, Bd = block_dynamics(rng, nx, nu, 10, spectral_radius)
    else:
        raise ValueError(dynamics)
    Q = np.eye(nx)
    R = 0.1 * np.eye(nu)
    P, Acon, F, E, l0, u0, K = condensed_mpc(Ad, Bd, Q, R, Q, N, umax)
    if extra_ineq:
        n = P.shape[0]
        rng2 = rng_for(workload_id, 1)
        G = rng2.standard_normal((extra_ineq, n)) / np.sqrt(n)
        h = rng2.uniform(1.0, 2.0, extra_ineq)
        Acon = np.vstack([Acon, G])
        E = np.vstack([E, np.zeros((extra_ineq, nx))])
        l0 = np.concatenate([l0, -np.inf * np.ones(extra_ineq)])
        u0 = np.concatenate([u0, h])
    return ParametricQP(P=P, A=Acon, F=F, E=E, l0=l0, u0=u0, Ad=Ad, Bd=Bd, K=K, N=N, name=name,
                        meta=dict(nx=nx, nu=nu, N=N, umax=umax, dynamics=dynamics,
                                  spectral_radius=spectral_radius, extra_ineq=extra_ineq,
                                  workload_id=workload_id))


def initial_states(nx: int, count: int, workload_id: int, sub_id: int = 2, std: float = 1.0):
    """count seeded initial states x0 ~ N(0, std^2), shape (count, nx)."""
    return std * rng_for(workload_id, sub_id).standard_normal((count, nx))


# ---------------------------------------------------------------------------
# the five synthetic workloads
# ---------------------------------------------------------------------------

SIGMA = 1e-6
RHO_BANK = (0.1, 1.0, 10.0)


def small_mpc() -> ParametricQP:
    """nx=6, nu=2, N=10: n = m = 20, |u| <= 1, spectral radius 1.05."""
    return mpc_problem(6, 2, 10, 1.0, 0, name="mpc_nx6_nu2_N10")


def sweep_mpc(nu: int) -> ParametricQP:
    """Horizon 40, nx = 3 nu, |u| <= 1: n = m = 40 nu."""
    return mpc_problem(3 * nu, nu, 40, 1.0, 100 + nu, name=f"mpc_nx{3*nu}_nu{nu}_N40")


def batched_mpc() -> ParametricQP:
    """nx=60, nu=20, N=40: n = m = 800 (many QPs share it, each with its own x0)."""
    return mpc_problem(60, 20, 40, 1.0, 2, name="mpc_nx60_nu20_N40")


def humanoid_mpc() -> ParametricQP:
    """nx=70, nu=30, N=20, block dynamics (radius 1.0), |u|<=50 + 400 dense rows: m=1000."""
    return mpc_problem(70, 30, 20, 50.0, 3, dynamics="block", spectral_radius=1.0,
                       extra_ineq=400, name="humanoid_nx70_nu30_N20_g400")


def served_family(which: int) -> ParametricQP:
    """The three resident families of the served stream: n = 80, 600, 1600."""
    if which == 0:
        return mpc_problem(12, 4, 20, 1.0, 40, name="mpc_nx12_nu4_N20")
    if which == 1:
        return humanoid_mpc()
    if which == 2:
        return mpc_problem(120, 40, 40, 1.0, 42, name="mpc_nx120_nu40_N40")
    raise ValueError(which)


def poisson_arrivals(rate_hz: float, duration_s: float, mix=(0.6, 0.3, 0.1), workload_id: int = 4,
                     sub_id: int = 5):
    """Arrival times (s) and family indices of a Poisson request stream."""
    rng = rng_for(workload_id, sub_id)
    times = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        times.append(t)
    times = np.asarray(times)
    fam = rng.choice(len(mix), size=len(times), p=np.asarray(mix) / np.sum(mix))
    return times, fam


# ---------------------------------------------------------------------------
# initial-state scale: big enough that the control limits bind
# ---------------------------------------------------------------------------

#: peak unconstrained LQR control / limit for the |u| <= 1 workloads
LIMIT_RATIO = 4.0
#: same for the humanoid-sized workload (|u| <= 50 plus dense rows)
LIMIT_RATIO_HUMANOID = 1.0


def x0_scale(pq: ParametricQP, ratio: float, draws: int = 64, sub_id: int = 9) -> float:
    """Standard deviation s of x0 = s N(0, I) that activates the control limits.

    In the paper's random-MPC runs (Sec. V-B) the initial states are chosen big
    enough that the control limits bind over a substantial part of the
    trajectory.  Along the
    unconstrained LQR rollout the controls are u_k = -K Abar^k x0, i.e. the
    rows E x0 of the limit rows; s is set so that the median over ``draws``
    seeded unit draws of max |E x0| / limit equals ``ratio``.
    """
    X = rng_for(pq.meta["workload_id"], sub_id).standard_normal((draws, pq.nx))
    box = np.isfinite(pq.l0) & np.isfinite(pq.u0) & (np.abs(pq.E).sum(1) > 0)
    r = np.max(np.abs(X @ pq.E[box].T) / pq.u0[box][None, :], axis=1)
    return float(ratio / np.median(r))


def default_x0_std(pq: ParametricQP) -> float:
    ratio = LIMIT_RATIO_HUMANOID if pq.meta.get("extra_ineq", 0) else LIMIT_RATIO
    return x0_scale(pq, ratio)


def workload(name: str, count: int = 1, x0_std: float | None = None):
    """(ParametricQP, x0 batch of shape (count, nx), x0 std) for a named workload.

    Names: "small" (n=m=20), "sweep<nu>" (n=m=40 nu), "batched" (n=m=800),
    "humanoid" (n=600, m=1000), "family<k>" (served families k=0,1,2).
    ``x0_std=None`` applies the limit-activation rule; pass 1.0 for the
    unscaled N(0,1) draws.
    """
    if name == "small":
        pq = small_mpc()
    elif name.startswith("sweep"):
        pq = sweep_mpc(int(name[5:]))
    elif name == "batched":
        pq = batched_mpc()
    elif name == "humanoid":
        pq = humanoid_mpc()
    elif name.startswith("family"):
        pq = served_family(int(name[6:]))
    else:
        raise ValueError(name)
    s = default_x0_std(pq) if x0_std is None else float(x0_std)
    X0 = initial_states(pq.nx, count, pq.meta["workload_id"], sub_id=2, std=s)
    return pq, X0, s


def disturbances(pq: ParametricQP, steps: int, std: float, sub_id: int = 3):
    """Closed-loop process noise w_t ~ N(0, std^2), shape (steps, nx)."""
    return std * rng_for(pq.meta["workload_id"], sub_id).standard_normal((steps, pq.nx))


def badly_scaled_qp(seed: int, n: int, m: int):
    """A dense QP whose variables and constraint rows span three orders of
    magnitude (row scales r, variable scales s in 10^U[-1.5, 1.5]):
    P = S (M M^T / n + I) S, A = R N S / sqrt(n), q = S g, and l <= A x <= u
    around A x_s (x_s = h / s) with widths proportional to r, so that about
    half the rows bind.  The entries of P and A span six orders of magnitude
    while x, A x and P x at the optimum stay below about 100, so that an
    absolute tolerance of 1e-3 is within FP32's reach once the problem is
    scaled.  Workload of the scaling tests (Algorithm 1's "Scale problem" step)."""
    rng = rng_for(90, seed)
    s = 10.0 ** rng.uniform(-1.5, 1.5, n)
    M = rng.standard_normal((n, n))
    P = (s[:, None] * (M @ M.T / n + np.eye(n))) * s[None, :]
    P = 0.5 * (P + P.T)
    r = 10.0 ** rng.uniform(-1.5, 1.5, m)
    A = r[:, None] * rng.standard_normal((m, n)) * s[None, :] / np.sqrt(n)
    q = s * rng.standard_normal(n)
    xs = rng.standard_normal(n) / s
    Ax = A @ xs
    l = Ax - r * rng.uniform(0.1, 1.0, m)
    u = Ax + r * rng.uniform(0.1, 1.0, m)
    return P, q, A, l, u
