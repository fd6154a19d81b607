"""Pins for the FP64 oracle: each checks it against something other than itself.

Pins (all CPU):
  * layer == the reordered three-step update (Sec. III-A, Eq. gpu_update vs
    Eqs. basic_lambda_update, basic_y_update, clamp) for random states;
  * layer iterates == standard ADMM iterates with mu (Sec. II-B, Eqs.
    Xbar_update .. lambda_update_gen) under the multiplier index shift, with a
    fixed rho and across a rho switch;
  * hand-derived optima of tiny QPs (tests/golden/hand_qps.json);
  * closed form x = -P^{-1} q without active constraints;
  * brute-force enumeration of all active sets for m <= 8;
  * KKT conditions of the reference optimum; fixed point of the layer there;
  * Cholesky / inverse against the library routine;
  * the penalty rule (Eq. rho_update) on cases whose answer is fixed by
    the formula's structure (balanced residuals, scaling, guards, ties);
  * planted mistakes (a flipped sign, a dropped term, a transposed block, a
    wrong multiplier index) are caught by the pins above;
  * the scaling step (Algorithm 1 "Scale problem", reading R10): a closed form
    for diagonal P, the optimum unchanged by the change of variables, the
    equilibration property, and the unscaled stop test on badly scaled QPs.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import relu_qp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_qp(seed, n, m, active=True, eq_rows=0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + 0.5 * np.eye(n)
    A = rng.standard_normal((m, n))
    q = rng.standard_normal(n) * (3.0 if active else 0.1)
    l = -rng.uniform(0.2, 1.0, m)
    u = rng.uniform(0.2, 1.0, m)
    if eq_rows:
        l[:eq_rows] = u[:eq_rows] = rng.uniform(-0.3, 0.3, eq_rows)
    return P, q, A, l, u


# ---------------------------------------------------------------------------
# layer algebra
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed,n,m,eq", [(0, 7, 5, 0), (1, 12, 20, 3), (2, 30, 9, 0)])
def test_layer_equals_reordered_three_step(seed, n, m, eq):
    P, q, A, l, u = random_qp(seed, n, m, eq_rows=eq)
    rng = np.random.default_rng(100 + seed)
    for rho in (0.1, 1.0, 10.0):
        rv = O.rho_vector(l, u, rho)
        W, Bop = O.relu_layer_weights(P, A, 1e-6, rv)
        b = Bop @ q
        for _ in range(5):
            x, z, lam = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
            v = O.relu_layer_step(W, b, np.concatenate([x, z, lam]), n, m, l, u)
            x2, z2, lam2 = O.admm_step_modified(P, q, A, l, u, 1e-6, rv, x, z, lam)
            ref = np.concatenate([x2, z2, lam2])
            assert np.max(np.abs(v - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))


def _shifted_compare(P, q, A, l, u, rho, iters, x0):
    n, m = P.shape[0], A.shape[0]
    z0 = A @ x0
    lay = O.layer_iterates(P, q, A, l, u, 1e-6, rho, iters, x0=x0, z0=z0, lam0=np.zeros(m))
    std = O.admm_iterates(P, q, A, l, u, 1e-6, rho, iters, x0=x0, z0=z0, lam0=np.zeros(m))
    rv = O.rho_vector(l, u, rho)
    worst = 0.0
    for v, (xs, zs, ls) in zip(lay, std):
        x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
        lam = O.std_multiplier(A, x, z, lam_l, rv)
        scale = 1 + max(np.max(np.abs(xs)), np.max(np.abs(ls)))
        worst = max(worst, np.max(np.abs(x - xs)) / scale, np.max(np.abs(z - zs)) / scale,
                    np.max(np.abs(lam - ls)) / scale)
    return worst


@pytest.mark.parametrize("seed,rho", [(3, 0.1), (4, 1.0), (5, 10.0)])
def test_layer_iterates_equal_standard_admm(seed, rho):
    P, q, A, l, u = random_qp(seed, 9, 6)
    x0 = np.random.default_rng(seed).standard_normal(9)
    assert _shifted_compare(P, q, A, l, u, rho, 200, x0) <= 1e-12


@pytest.mark.parametrize("seed,rho", [(3, 0.1), (4, 1.0), (5, 10.0)])
def test_layer_iterates_equal_standard_admm_with_equality_row(seed, rho):
    # The 1000x penalty of an equality row multiplies the rounding difference
    # between the explicit inverse (layer) and the solve (ADMM) into the
    # multiplier step every iteration, so the bound is looser; a formula
    # error would still show as an O(1) difference.
    P, q, A, l, u = random_qp(seed, 9, 6, eq_rows=1)
    x0 = np.random.default_rng(seed).standard_normal(9)
    assert _shifted_compare(P, q, A, l, u, rho, 200, x0) <= 1e-6


def test_layer_iterates_equal_standard_admm_across_rho_switch():
    """Rebase reading: after a switch the layer continues standard ADMM with the new rho."""
    P, q, A, l, u = random_qp(7, 10, 8)
    n, m = 10, 8
    rho1, rho2 = 0.1, 10.0
    rv1, rv2 = O.rho_vector(l, u, rho1), O.rho_vector(l, u, rho2)
    W1, B1 = O.relu_layer_weights(P, A, 1e-6, rv1)
    W2, B2 = O.relu_layer_weights(P, A, 1e-6, rv2)
    v = np.zeros(n + 2 * m)
    x, z, lam, mu = np.zeros(n), np.zeros(m), np.zeros(m), np.zeros(n)
    worst = 0.0
    for it in range(1, 121):
        rv, W, b = (rv1, W1, B1 @ q) if it <= 40 else (rv2, W2, B2 @ q)
        v = O.relu_layer_step(W, b, v, n, m, l, u)
        x, z, lam, mu, _ = O.admm_step_standard(P, q, A, l, u, 1e-6, rv, x, z, lam, mu)
        vx, vz, vl = v[:n], v[n:n + m], v[n + m:]
        lam_std = O.std_multiplier(A, vx, vz, vl, rv)
        worst = max(worst, np.max(np.abs(vx - x)), np.max(np.abs(lam_std - lam)))
        if it == 40:  # switch rho1 -> rho2 with the rebase of the layer multiplier
            v[n + m:] = lam_std - rv2 * (A @ vx - vz)
    assert worst <= 1e-11


# ---------------------------------------------------------------------------
# optimum pins
# ---------------------------------------------------------------------------

def _load_hand():
    with open(os.path.join(GOLDEN, "hand_qps.json")) as f:
        data = json.load(f)["problems"]
    out = []
    for p in data:
        l = np.array([-np.inf if v is None else v for v in p["l"]])
        u = np.array([np.inf if v is None else v for v in p["u"]])
        out.append((p["name"], np.array(p["P"]), np.array(p["q"]), np.array(p["A"]), l, u,
                    np.array(p["x"]), np.array(p["lam"])))
    return out


@pytest.mark.parametrize("case", _load_hand(), ids=lambda c: c[0])
def test_hand_derived_optima(case):
    name, P, q, A, l, u, x_star, lam_star = case
    r = O.solve(P, q, A, l, u, eps_abs=1e-9, max_iter=100000)
    assert r.status == "solved"
    assert np.max(np.abs(r.x - x_star)) <= 1e-6
    assert np.max(np.abs(r.lam - lam_star)) <= 1e-5
    ref = O.reference_solution(P, q, A, l, u)
    assert np.max(np.abs(ref["x"] - x_star)) <= 1e-9
    assert np.max(np.abs(ref["lam"] - lam_star)) <= 1e-8


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_unconstrained_closed_form(seed):
    rng = np.random.default_rng(seed)
    n, m = 15, 10
    M = rng.standard_normal((n, n))
    P = M @ M.T + np.eye(n)
    q = rng.standard_normal(n)
    A = rng.standard_normal((m, n))
    l = -np.inf * np.ones(m)
    u = np.inf * np.ones(m)
    r = O.solve(P, q, A, l, u, eps_abs=1e-10, max_iter=20000)
    x_cf = -np.linalg.solve(P, q)
    assert r.status == "solved"
    assert np.max(np.abs(r.x - x_cf)) <= 1e-8 * (1 + np.max(np.abs(x_cf)))
    assert np.max(np.abs(r.lam)) <= 1e-9


@pytest.mark.parametrize("seed,m", [(21, 4), (22, 6), (23, 8), (24, 7)])
def test_brute_force_active_set(seed, m):
    P, q, A, l, u = random_qp(seed, 6, m, eq_rows=1 if m > 5 else 0)
    bf = O.brute_force_qp(P, q, A, l, u)
    ref = O.reference_solution(P, q, A, l, u)
    assert np.max(np.abs(ref["x"] - bf["x"])) <= 1e-9 * (1 + np.max(np.abs(bf["x"])))
    r = O.solve(P, q, A, l, u, eps_abs=1e-9, max_iter=200000)
    assert np.max(np.abs(r.x - bf["x"])) <= 1e-6
    # at least one constraint is active, so the test is not the closed form again
    assert np.count_nonzero(np.abs(bf["lam"]) > 1e-8) >= 1


def test_reference_kkt_and_fixed_point_on_mpc():
    from workloads import mpc
    pq, X0, _ = mpc.workload("small", 3)
    for x0 in X0:
        q, l, u = pq.instance(x0)
        ref = O.reference_solution(pq.P, q, pq.A, l, u)
        assert ref["kkt"] <= 1e-9
        # fixed point: with z = Ax and lam' = lam* the layer maps v* onto itself
        rv = O.rho_vector(l, u, 1.0)
        W, Bop = O.relu_layer_weights(pq.P, pq.A, 1e-6, rv)
        x, lam = ref["x"], ref["lam"]
        z = np.minimum(np.maximum(pq.A @ x, l), u)
        v = np.concatenate([x, z, lam])
        v2 = O.relu_layer_step(W, Bop @ q, v, pq.n, pq.m, l, u)
        assert np.max(np.abs(v2 - v)) <= 1e-9 * (1 + np.max(np.abs(v)))


def test_cholesky_and_inverse_against_library():
    P, q, A, l, u = random_qp(31, 40, 30)
    rv = O.rho_vector(l, u, 1.0)
    D, L = O.kkt_inverse(P, A, 1e-6, rv)
    K = O.kkt_matrix(P, A, 1e-6, rv)
    assert np.linalg.norm(L @ L.T - K) / np.linalg.norm(K) <= 1e-13
    Dlib = np.linalg.inv(K)
    assert np.max(np.abs(D - Dlib)) <= 1e-11 * np.max(np.abs(Dlib))


def test_equality_rows_get_scaled_penalty():
    l = np.array([0.0, 1.0, -np.inf])
    u = np.array([0.0, 2.0, 3.0])
    rv = O.rho_vector(l, u, 0.5)
    assert rv.tolist() == [500.0, 0.5, 0.5]


# ---------------------------------------------------------------------------
# penalty rule
# ---------------------------------------------------------------------------

def _res(rp, rd, Ax=1.0, z=1.0, Px=1.0, Atl=1.0, qn=1.0):
    return dict(r_prim=rp, r_dual=rd, Ax=Ax, z=z, Px=Px, Atl=Atl, q=qn)


def test_rho_rule_structure():
    # balanced normalised residuals keep rho
    assert O.rho_estimate(0.7, _res(1e-2, 1e-2)) == pytest.approx(0.7)
    # 100x larger primal residual -> rho grows by sqrt(100)
    assert O.rho_estimate(1.0, _res(1.0, 1e-2)) == pytest.approx(10.0)
    # normalisers enter as a ratio: scaling both by the same factor changes nothing
    a = O.rho_estimate(1.0, _res(3e-3, 5e-4, Ax=2.0, z=7.0, Px=5.0, Atl=1.0, qn=0.1))
    b = O.rho_estimate(1.0, _res(3e-3, 5e-4, Ax=20.0, z=70.0, Px=50.0, Atl=10.0, qn=1.0))
    assert a == pytest.approx(b)
    # floors of 1e-4 bind when every norm is tiny
    assert O.rho_estimate(1.0, _res(1e-6, 1e-6, 0, 0, 0, 0, 0)) == pytest.approx(1.0)
    # guards: zero residual keeps the index
    assert math.isnan(O.rho_estimate(1.0, _res(0.0, 1.0)))
    assert O.nearest_rho_index((0.1, 1.0, 10.0), float("nan"), 1) == 1


def test_nearest_rho_index():
    bank = (0.1, 1.0, 10.0)
    assert O.nearest_rho_index(bank, 0.2, 2) == 0
    assert O.nearest_rho_index(bank, 0.5, 0) == 1
    assert O.nearest_rho_index(bank, 5.0, 0) == 2
    assert O.nearest_rho_index(bank, 1e6, 0) == 2
    # geometric midpoint is a tie in log distance -> lower index
    assert O.nearest_rho_index(bank, math.sqrt(0.1 * 1.0), 2) == 0


def test_algorithm1_switches_to_balance_and_returns_std_multiplier():
    P, q, A, l, u = random_qp(41, 20, 15)
    r = O.solve(P, q, A, l, u, eps_abs=1e-7, rho0=0.1, rho_bank=(0.001, 0.01, 0.1, 1.0, 10.0, 100.0))
    assert r.status == "solved"
    # returned multiplier satisfies stationarity to the tolerance
    assert np.max(np.abs(P @ r.x + q + A.T @ r.lam)) <= 1e-7
    assert r.iters % 25 == 0


def test_warm_start_at_optimum_converges_at_first_check():
    P, q, A, l, u = random_qp(42, 12, 9)
    ref = O.reference_solution(P, q, A, l, u)
    r = O.solve(P, q, A, l, u, eps_abs=1e-6, x_warm=ref["x"], lam_warm=ref["lam"])
    assert r.status == "solved" and r.iters == 25
    assert np.max(np.abs(r.x - ref["x"])) <= 1e-6


# ---------------------------------------------------------------------------
# planted mistakes: each mutation of the layer must break a pin above
# ---------------------------------------------------------------------------

def _mutants():
    def flip_wzl(W, Bop, n, m, A, rv):
        W = W.copy()
        W[n:n + m, n + m:] *= -1.0
        return W, Bop

    def drop_rinv(W, Bop, n, m, A, rv):
        W = W.copy()
        W[n:n + m, n + m:] -= np.diag(1.0 / rv)
        return W, Bop

    def wrong_rho_in_lam_row(W, Bop, n, m, A, rv):
        W = W.copy()
        W[n + m:, :n] = A       # rho G -> G
        return W, Bop

    def bias_sign(W, Bop, n, m, A, rv):
        return W, -Bop

    def two_to_one(W, Bop, n, m, A, rv):
        W = W.copy()
        W[:n, n:n + m] *= 0.5   # 2 D G^T rho -> D G^T rho
        return W, Bop
    return [flip_wzl, drop_rinv, wrong_rho_in_lam_row, bias_sign, two_to_one]


@pytest.mark.parametrize("mutant", _mutants(), ids=lambda f: f.__name__)
def test_planted_layer_mistakes_are_caught(mutant):
    P, q, A, l, u = random_qp(51, 8, 6)
    n, m = 8, 6
    rv = O.rho_vector(l, u, 2.5)      # rho != 1 so that rho G differs from G
    W, Bop = O.relu_layer_weights(P, A, 1e-6, rv)
    Wm, Bm = mutant(W, Bop, n, m, A, rv)
    rng = np.random.default_rng(0)
    x, z, lam = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
    v = O.relu_layer_step(Wm, Bm @ q, np.concatenate([x, z, lam]), n, m, l, u)
    ref = np.concatenate(O.admm_step_modified(P, q, A, l, u, 1e-6, rv, x, z, lam))
    assert np.max(np.abs(v - ref)) > 1e-6


def test_planted_index_shift_mistake_is_caught():
    """Comparing layer lam' directly with standard lam (no shift) must fail."""
    P, q, A, l, u = random_qp(52, 9, 6)
    n, m = 9, 6
    lay = O.layer_iterates(P, q, A, l, u, 1e-6, 1.0, 30)
    std = O.admm_iterates(P, q, A, l, u, 1e-6, 1.0, 30)
    diff = max(np.max(np.abs(v[n + m:] - s[2])) for v, s in zip(lay, std))
    assert diff > 1e-6


# ---------------------------------------------------------------------------
# Algorithm 1 "Scale problem": modified Ruiz equilibration (reading R10)
# ---------------------------------------------------------------------------

def test_ruiz_diagonal_closed_form():
    """P diagonal, no constraints: one iteration scales every variable by
    1/sqrt(p_j), making the scaled P the identity before the cost scale
    c = 1 / max(1, |q / sqrt(p)|_inf)."""
    p = np.array([4.0, 0.25, 9.0, 1.0])
    q = np.array([1.0, -3.0, 0.5, 2.0])
    D, E, c, Pb, Ab, qb = O.ruiz_scaling(np.diag(p), np.zeros((0, 4)), q, iters=1)
    assert E.size == 0 and Ab.shape == (0, 4)
    np.testing.assert_allclose(D, 1.0 / np.sqrt(p), rtol=1e-15)
    c_expected = 1.0 / max(1.0, np.max(np.abs(q / np.sqrt(p))))
    assert c == pytest.approx(c_expected, rel=1e-15)
    np.testing.assert_allclose(Pb, c_expected * np.eye(4), atol=1e-15)
    np.testing.assert_allclose(qb, c_expected * q / np.sqrt(p), rtol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_ruiz_keeps_the_optimum(seed):
    """The scaled problem's optimum, mapped back (x = D xb, lam = E lamb / c),
    is the original problem's optimum: scaling is a change of variables."""
    from workloads import mpc
    P, q, A, l, u = mpc.badly_scaled_qp(seed, 14, 9)
    D, E, c, Pb, Ab, qb = O.ruiz_scaling(P, A, q, iters=10)
    ref = O.reference_solution(P, q, A, l, u)
    refb = O.reference_solution(Pb, qb, Ab, E * l, E * u)
    assert ref["kkt"] < 1e-7 and refb["kkt"] < 1e-7
    np.testing.assert_allclose(D * refb["x"], ref["x"], atol=1e-7 * (1 + np.abs(ref["x"]).max()))
    np.testing.assert_allclose(E * refb["lam"] / c, ref["lam"], atol=1e-6 * (1 + np.abs(ref["lam"]).max()))


def test_ruiz_equilibrates_the_kkt_matrix():
    """The iterations drive the infinity norms of the columns of the scaled KKT
    matrix [[Pb, Ab^T], [Ab, 0]] towards 1: a spread of more than 1000 between
    the largest and the smallest shrinks below 1.2 in 25 iterations (the cost
    step rescales P after each one, so the norms approach 1 gradually)."""
    from workloads import mpc
    P, q, A, l, u = mpc.badly_scaled_qp(3, 20, 12)
    before = np.abs(np.block([[P, A.T], [A, np.zeros((12, 12))]])).max(axis=0)
    D, E, c, Pb, Ab, qb = O.ruiz_scaling(P, A, np.zeros(20), iters=25)
    K = np.block([[Pb, Ab.T], [Ab, np.zeros((12, 12))]])
    after = np.abs(K).max(axis=0)
    assert before.max() / before.min() > 1e3
    assert after.max() / after.min() < 1.2


def test_scaled_solve_meets_the_unscaled_stop_test_and_helps():
    """Badly scaled QPs: without scaling ADMM does not reach eps = 1e-3 in 4000
    layers; with it, it stops at a point whose original-problem residuals meet
    eps and which is within 1e-3 of the optimum."""
    from workloads import mpc
    P, q, A, l, u = mpc.badly_scaled_qp(0, 40, 30)
    plain = O.solve(P, q, A, l, u, eps_abs=1e-3, max_iter=4000)
    r = O.solve_scaled(P, q, A, l, u, scaling_iters=10, eps_abs=1e-3, max_iter=4000)
    ref = O.reference_solution(P, q, A, l, u)
    res = O.residuals(P, q, A, r.x, r.z, r.lam)
    assert plain.status == "max_iter"
    assert r.status == "solved" and r.iters < 2000
    assert res["r_prim"] <= 1e-3 and res["r_dual"] <= 1e-3
    assert np.max(np.abs(r.x - ref["x"])) <= 1e-3


def test_fixed_scaling_is_the_computed_one_for_the_setup_q():
    """solve_scaled with the (D, E, c) that ruiz_scaling returns for this q is the
    same computation as letting it scale: identical iterates and result."""
    from workloads import mpc
    P, q, A, l, u = mpc.badly_scaled_qp(1, 30, 20)
    D, E, c, *_ = O.ruiz_scaling(P, A, q, 10)
    a = O.solve_scaled(P, q, A, l, u, scaling_iters=10, eps_abs=1e-3, max_iter=2000)
    b = O.solve_scaled(P, q, A, l, u, scaling=(D, E, c), eps_abs=1e-3, max_iter=2000)
    assert a.iters == b.iters and a.status == b.status
    assert np.max(np.abs(a.x - b.x)) <= 1e-12 * max(1.0, np.max(np.abs(a.x)))
