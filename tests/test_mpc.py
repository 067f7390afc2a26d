"""Pins of the host-side model predictive controller (paper: section "Model
Predictive Control of WECs"): the matrix exponential and the first-order-hold
discretisation against library and numerical integration, the prediction
matrices against marching the discrete model, the objective weight against
its defining sum, the box QP against brute-force enumeration of its KKT points,
the free-decay identification against a closed-form damped oscillation, and
the closed loop on the linear plant (absorbs energy, respects the force limit)."""
import math

import numpy as np
import pytest

from paper_2206_07732_gb300 import mpc

scipy_linalg = pytest.importorskip("scipy.linalg")
scipy_integrate = pytest.importorskip("scipy.integrate")


def test_expm_matches_library():
    rng = np.random.default_rng(0)
    for s in (0.01, 1.0, 30.0):
        A = s * rng.standard_normal((4, 4))
        assert np.allclose(mpc.expm(A), scipy_linalg.expm(A), rtol=1e-11, atol=1e-12 * np.max(np.abs(scipy_linalg.expm(A))))


def test_foh_step_equals_integrated_plant():
    # one control step of the continuous plant with u, v linear in time equals
    # A_d X + B_d du + F_d dv (Eq. disc_SS_sysa)
    m, kh, cr, dt = 410.0, 1025.0 * 9.81 * 1.0, 180.0, 0.05
    A, B = mpc.continuous_model(m, kh, cr)
    Ad, Bd, Fd, Cd = mpc.foh_model(A, B, dt)
    x0 = np.array([0.03, -0.1])
    u0, u1, v0, v1 = 0.7, -1.3, 2.1, 0.4
    rhs = lambda t, x: A @ x + B[:, 0] * (u0 + (u1 - u0) * t / dt + v0 + (v1 - v0) * t / dt)
    sol = scipy_integrate.solve_ivp(rhs, (0.0, dt), x0, rtol=1e-12, atol=1e-14)
    X = Ad @ np.array([x0[0], x0[1], u0, v0]) + Bd[:, 0] * (u1 - u0) + Fd[:, 0] * (v1 - v0)
    assert np.allclose(X[:2], sol.y[:, -1], rtol=1e-9, atol=1e-12)
    assert X[2] == pytest.approx(u1) and X[3] == pytest.approx(v1)
    assert np.array_equal(Cd @ X, X[[0, 1, 2]])


def test_prediction_matrices_equal_marching():
    m, kh, cr, dt, Np = 300.0, 8000.0, 90.0, 0.05, 12
    Ad, Bd, Fd, Cd = mpc.foh_model(*mpc.continuous_model(m, kh, cr), dt)
    P, Ju, Jv = mpc.prediction_matrices(Ad, Bd, Fd, Cd, Np)
    rng = np.random.default_rng(1)
    X = rng.standard_normal(4)
    du, dv = rng.standard_normal(Np), rng.standard_normal(Np)
    Z = []
    x = X.copy()
    for i in range(Np):
        x = Ad @ x + Bd[:, 0] * du[i] + Fd[:, 0] * dv[i]
        Z.append(Cd @ x)
    assert np.allclose(P @ X + Ju @ du + Jv @ dv, np.concatenate(Z), rtol=1e-12, atol=1e-12)


def test_energy_weight_is_the_trapezoid_sum():
    rng = np.random.default_rng(2)
    Np = 7
    Z = rng.standard_normal(3 * Np)
    Q = mpc.energy_weight(Np)
    zd, u = Z[1::3], Z[2::3]
    assert 0.5 * Z @ Q @ Z == pytest.approx(np.sum(u[:-1] * zd[:-1]) + 0.5 * u[-1] * zd[-1], rel=1e-13)


def _brute_box_qp(H, f, lo, hi):
    # every assignment of each variable to its lower bound, upper bound or free
    import itertools
    best, xbest = None, None
    n = len(f)
    for pat in itertools.product((0, 1, 2), repeat=n):
        x = np.where(np.array(pat) == 0, lo, np.where(np.array(pat) == 1, hi, 0.0))
        F = np.array(pat) == 2
        if F.any():
            x = x.copy()
            x[F] = np.linalg.solve(H[np.ix_(F, F)], -(f[F] + H[np.ix_(F, ~F)] @ x[~F]))
        if np.any(x < lo - 1e-12) or np.any(x > hi + 1e-12):
            continue
        val = 0.5 * x @ H @ x + f @ x
        if best is None or val < best:
            best, xbest = val, x
    return xbest


def test_box_qp_equals_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(40):
        n = 4
        R = rng.standard_normal((n, n))
        H = R @ R.T + 0.1 * np.eye(n)
        f = 3.0 * rng.standard_normal(n)
        lo, hi = -rng.uniform(0.1, 1.0, n), rng.uniform(0.1, 1.0, n)
        x = mpc.box_qp(H, f, lo, hi)
        assert np.allclose(x, _brute_box_qp(H, f, lo, hi), atol=1e-9)


def test_free_decay_identification():
    m, kh, zeta = 420.0, 10055.0, 0.08
    wn = math.sqrt(kh / m)
    wd = wn * math.sqrt(1 - zeta ** 2)
    t = np.arange(0.0, 8.0, 1e-3)
    z = 0.02 * np.exp(-zeta * wn * t) * np.cos(wd * t)
    m_eff, c_r, wn_i, zeta_i = mpc.identify_free_decay(t, z, kh)
    assert m_eff == pytest.approx(m, rel=2e-3)
    assert zeta_i == pytest.approx(zeta, rel=2e-2)
    assert c_r == pytest.approx(2 * zeta * wn * m, rel=2e-2)


@pytest.mark.parametrize("f_max", [2000.0, 200.0])
def test_closed_loop_absorbs_energy_within_the_force_limit(f_max):
    # linear plant driven by a regular wave's excitation, the MPC force applied
    # with first-order hold, fine time steps: positive absorbed energy, |F| <= f_max
    m, kh, cr = 410.0, 1025.0 * 9.81, 120.0
    T, Fa = 1.6, 400.0
    w = 2 * math.pi / T
    dt_p, sub = 0.05, 50
    Np = math.ceil(T / dt_p)
    ctl = mpc.MPC(m, kh, cr, dt_p, Np, lam1=2.0, lam2=0.2, f_max=f_max)
    A, B = mpc.continuous_model(m, kh, cr)
    h = dt_p / sub
    Ad, Bd, Fd, _ = mpc.foh_model(A, B, h)
    x = np.zeros(2)
    F_now, E = 0.0, 0.0
    fexc = lambda t: Fa * math.cos(w * t)
    for k in range(int(20 * T / dt_p)):
        t0 = k * dt_p
        U = ctl.solve(x[0], x[1], F_now, fexc(t0), [fexc(t0 + (i + 1) * dt_p) for i in range(Np)])
        F_next = U[0]
        assert abs(F_next) <= f_max * (1 + 1e-9)
        ramp = ctl.ramp(F_now, F_next, sub)
        for i in range(sub):
            tt = t0 + i * h
            u0, u1 = ramp[i] / m, (ramp[i + 1] if i + 1 < sub else F_next) / m
            v0, v1 = fexc(tt) / m, fexc(tt + h) / m
            X = Ad @ np.array([x[0], x[1], u0, v0]) + Bd[:, 0] * (u1 - u0) + Fd[:, 0] * (v1 - v0)
            zd0 = x[1]
            x = X[:2]
            E -= 0.5 * (u0 * zd0 + u1 * x[1]) * m * h  # absorbed energy: -int F zd dt
        F_now = F_next
    print(f"f_max {f_max}: absorbed {E:.1f} J/m over 20 periods")
    assert E > 0.0


# ---- the path constraints of Eq. path_constr and the AR forecast (section "AR predictions")

def test_general_qp_equals_brute_force_kkt():
    # the interior-point QP (polished on its active set) against the best KKT
    # point found by enumerating every active set of small random problems
    import itertools
    rng = np.random.default_rng(11)
    for _ in range(120):
        n, m = int(rng.integers(2, 6)), int(rng.integers(1, 9))
        A = rng.standard_normal((n, n))
        H = A @ A.T + 0.1 * np.eye(n)
        f = rng.standard_normal(n)
        G = rng.standard_normal((m, n))
        h = np.abs(rng.standard_normal(m)) + 0.1
        x = mpc.qp_ineq(H, f, G, h)
        best = None
        for k in range(0, min(n, m) + 1):
            for S in itertools.combinations(range(m), k):
                S = list(S)
                K = np.block([[H, G[S].T], [G[S], np.zeros((k, k))]])
                try:
                    sol = np.linalg.solve(K, np.concatenate([-f, h[S]]))
                except np.linalg.LinAlgError:
                    continue
                xs, la = sol[:n], sol[n:]
                if np.all(G @ xs <= h + 1e-9) and np.all(la >= -1e-9):
                    v = 0.5 * xs @ H @ xs + f @ xs
                    if best is None or v < best[0]:
                        best = (v, xs)
        assert np.max(np.abs(x - best[1])) <= 1e-9 * (1.0 + np.max(np.abs(best[1])))


def test_general_qp_on_a_box_equals_the_box_qp():
    rng = np.random.default_rng(12)
    for _ in range(20):
        n = 8
        A = rng.standard_normal((n, n))
        H = A @ A.T + 0.5 * np.eye(n)
        f = 5.0 * rng.standard_normal(n)
        lo, hi = -np.ones(n), np.ones(n)
        xb = mpc.box_qp(H, f, lo, hi)
        xq = mpc.qp_ineq(H, f, np.vstack([np.eye(n), -np.eye(n)]), np.concatenate([hi, -lo]))
        assert np.max(np.abs(xb - xq)) <= 1e-9


def test_ar_fit_recovers_a_noise_free_ar3():
    # a record generated by an AR(3) recursion is fitted back exactly
    a = np.array([1.2, -0.5, 0.1])
    x = [1.0, -0.3, 0.7]
    for _ in range(60):
        x.append(a @ np.array(x[-1:-4:-1]))
    assert np.allclose(mpc.ar_fit(x, 3), a, rtol=0, atol=1e-9)


def test_ar_predicts_sums_of_sinusoids_exactly():
    # K sinusoids sampled at a fixed rate obey a linear recurrence of order 2 K
    # (each cos(w t + p) satisfies x_t = 2 cos(w dt) x_{t-1} - x_{t-2}): AR(2 K)
    # continues them without error
    t = np.arange(300) * 0.05
    for comps in ([(2.0, 0.3, 1.0)], [(2.0, 0.3, 1.0), (3.1, -1.0, 0.5)], [(1.5, 0.0, 1.0), (2.7, 2.0, 0.3), (4.2, 1.0, 0.2)]):
        x = sum(a * np.cos(w * t + p) for w, p, a in comps)
        k = 2 * len(comps)
        pred = mpc.ar_predict(x[:160], mpc.ar_fit(x[:160], k), 40)
        assert np.max(np.abs(pred - x[160:200])) <= 1e-7


def _plant(m, kh, cr, dt_p, sub):
    A, B = mpc.continuous_model(m, kh, cr)
    return mpc.foh_model(A, B, dt_p / sub)


def test_mpc_respects_displacement_and_velocity_bounds():
    # with the z, zd rows of Eq. path_constr the predicted trajectory stays in
    # the bounds; with bounds that never bind the solution is the box QP's
    m, kh, cr, dt_p = 410.0, 1025.0 * 9.81, 120.0, 0.05
    Np = 32
    rng = np.random.default_rng(13)
    free = mpc.MPC(m, kh, cr, dt_p, Np, lam1=2.0, lam2=0.2, f_max=2000.0)
    loose = mpc.MPC(m, kh, cr, dt_p, Np, lam1=2.0, lam2=0.2, f_max=2000.0, z_lim=(-10.0, 10.0), zd_lim=(-50.0, 50.0))
    tight = mpc.MPC(m, kh, cr, dt_p, Np, lam1=2.0, lam2=0.2, f_max=2000.0, z_lim=(-0.02, 0.02), zd_lim=(-0.08, 0.08))
    for _ in range(10):
        z, zd = 0.01 * rng.standard_normal(), 0.03 * rng.standard_normal()
        F_now = 200.0 * rng.standard_normal()
        t = np.arange(Np + 1) * dt_p
        fe = 800.0 * np.cos(2 * math.pi / 1.6 * t + rng.uniform(0, 6))
        Uf = free.solve(z, zd, F_now, fe[0], fe[1:])
        Ul = loose.solve(z, zd, F_now, fe[0], fe[1:])
        assert np.max(np.abs(Uf - Ul)) <= 1e-6 * (1.0 + np.max(np.abs(Uf)))
        Ut = tight.solve(z, zd, F_now, fe[0], fe[1:])
        pred = tight.predicted(z, zd, F_now, fe[0], fe[1:])
        assert np.all(np.abs(Ut) <= 2000.0 * (1 + 1e-9))
        # (a bound the initial state already violates cannot hold at step 1)
        zz = pred[1:, 0] if abs(z) > 0.02 else pred[:, 0]
        assert np.max(np.abs(zz)) <= 0.02 + 1e-8 or abs(z) > 0.02
        assert np.max(np.abs(pred[1:, 1])) <= 0.08 + 1e-8 or abs(zd) > 0.08


def test_closed_loop_with_ar_forecast_and_path_bounds():
    # the linear plant in an irregular sea (three components), the MPC fed (a)
    # the exact future excitation, (b) an AR(5) forecast fitted to the last two
    # peak periods of past excitation at the control rate (section "AR
    # predictions"), both with a displacement bound: energy is absorbed in both,
    # the forecast keeps most of it, the force limit holds, and the bound holds
    # at the control instants up to what the model cannot see
    m, kh, cr = 410.0, 1025.0 * 9.81, 120.0
    dt_p, sub, Tp = 0.05, 25, 1.6
    Np = math.ceil(Tp / dt_p)
    comps = [(2 * math.pi / 1.6, 0.0, 300.0), (2 * math.pi / 1.35, 1.1, 150.0), (2 * math.pi / 1.9, 2.3, 120.0)]
    fexc = lambda tt: sum(a * math.cos(w * tt + p) for w, p, a in comps)
    Ad, Bd, Fd, _ = _plant(m, kh, cr, dt_p, sub)
    h = dt_p / sub
    energy = {}
    for mode in ("exact", "ar"):
        ctl = mpc.MPC(m, kh, cr, dt_p, Np, lam1=2.0, lam2=0.2, f_max=600.0, z_lim=(-0.06, 0.06))
        fc = mpc.ArForecaster(order=5, window=int(2 * Tp / dt_p))
        x = np.zeros(2)
        F_now, E, zmax = 0.0, 0.0, 0.0
        for k in range(int(40 * Tp / dt_p)):
            t0 = k * dt_p
            fc.push(fexc(t0))
            if mode == "ar" and fc.ready():
                fut = fc.predict(Np)
            else:
                fut = [fexc(t0 + (i + 1) * dt_p) for i in range(Np)]
            F_next = float(ctl.solve(x[0], x[1], F_now, fexc(t0), fut)[0])
            assert abs(F_next) <= 600.0 * (1 + 1e-9)
            ramp = ctl.ramp(F_now, F_next, sub)
            for i in range(sub):
                tt = t0 + i * h
                u0, u1 = ramp[i] / m, (ramp[i + 1] if i + 1 < sub else F_next) / m
                v0, v1 = fexc(tt) / m, fexc(tt + h) / m
                X = Ad @ np.array([x[0], x[1], u0, v0]) + Bd[:, 0] * (u1 - u0) + Fd[:, 0] * (v1 - v0)
                zd0 = x[1]
                x = X[:2]
                E -= 0.5 * (u0 * zd0 + u1 * x[1]) * m * h
            F_now = F_next
            if k * dt_p > 10 * Tp:
                zmax = max(zmax, abs(x[0]))
        energy[mode] = E
        print(f"{mode}: absorbed {E:.1f} J/m, max |z| {zmax:.4f} m")
        assert zmax <= 0.06 * 1.05
    assert energy["exact"] > 0.0 and energy["ar"] > 0.7 * energy["exact"]
