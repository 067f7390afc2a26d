"""Host-side model predictive control of the heaving body's PTO force (paper:
section "Model Predictive Control of WECs" and its subsections on device
constraints and regularisation).  Small dense numpy code outside the GPU path:
one quadratic program per control interval.

Plant model (section "Linear potential theory-based WEC dynamical model", with
no radiation states: the radiation force is a linear damping c_r identified,
together with the effective mass, from a free-decay run of the tank itself; the
infinite-frequency added mass is folded into that effective mass):

    m_eff zdd = -k_h z - c_r zd + F_exc + F_PTO,     u = F_PTO / m_eff,  v = F_exc / m_eff

k_h = rho_w g W is the hydrostatic stiffness of the box per unit span.  The
first-order-hold discretisation (Eqs. disc_SS_sysa / disc_SS_sysb) augments the
state with u and v: X_d = [z, zd, u, v], and the inputs are their increments
over one control step dt_p.  Over N_p steps the outputs Z = [z, zd, u] stack
into Z = P X_d + J_u du + J_v dv (Eq. output_pred_vector).

Objective J_3 (Eqs. J1, J2, J3): the trapezoidal absorbed energy
sum u zd (J_1 = Z^T Q Z / 2) plus lam1 ||du||^2 plus lam2 ||u||^2, minimised
over the force sequence U = (u(k+1) .. u(k+N_p)) -- du = D U - e_1 u(k) -- under
the path constraints of Eq. path_constr: the force limit |F_PTO| <= f_max, a box
on U, and optionally bounds on the predicted displacement and velocity, which
are linear in U through the prediction (section "Including device/path
constraints in MPC").  The box QP is solved by a projected Newton method, the QP
with displacement / velocity rows by a primal-dual interior-point method.

Excitation forecast: the incident wave is known analytically (the tank's own
Airy components), F_exc(t) = k_h eta(x_B, t) (linear Froude-Krylov with a
hydrostatic gain), or forecast by an autoregressive model (section "AR
predictions"): AR(p) coefficients fitted by least squares to the last samples
of the excitation at the control rate, then the model run forward over the
horizon.
"""
from __future__ import annotations

import math

import numpy as np


def expm(A):
    """Matrix exponential by scaling and squaring of a Taylor series (small,
    well-scaled matrices)."""
    A = np.asarray(A, dtype=np.float64)
    nrm = np.max(np.sum(np.abs(A), axis=1))
    s = max(0, int(math.ceil(math.log2(nrm))) + 1) if nrm > 0.5 else 0
    X = A / (2.0 ** s)
    E = np.eye(A.shape[0])
    T = np.eye(A.shape[0])
    for k in range(1, 20):
        T = T @ X / k
        E = E + T
    for _ in range(s):
        E = E @ E
    return E


def continuous_model(m_eff, k_h, c_r):
    """A_c, B_c of the heave model with state [z, zd] and input u = F / m_eff."""
    A = np.array([[0.0, 1.0], [-k_h / m_eff, -c_r / m_eff]])
    B = np.array([[0.0], [1.0]])
    return A, B


def foh_model(A, B, dt):
    """First-order-hold discretisation (Eqs. disc_SS_sysa, uc_interpolation):
    returns A_d, B_d, F_d, C_d for the state [X_c, u, v]."""
    n = A.shape[0]
    phi = expm(dt * A)
    Ai = np.linalg.inv(A)
    ups = Ai @ (phi - np.eye(n)) @ B
    lam = Ai @ (ups - dt * B) / dt
    Ad = np.zeros((n + 2, n + 2))
    Ad[:n, :n] = phi
    Ad[:n, n:n + 1] = ups
    Ad[:n, n + 1:n + 2] = ups
    Ad[n, n] = 1.0
    Ad[n + 1, n + 1] = 1.0
    Bd = np.vstack([lam, [[1.0]], [[0.0]]])
    Fd = np.vstack([lam, [[0.0]], [[1.0]]])
    Cd = np.zeros((3, n + 2))
    Cd[0, 0] = 1.0
    Cd[1, 1] = 1.0
    Cd[2, n] = 1.0
    return Ad, Bd, Fd, Cd


def prediction_matrices(Ad, Bd, Fd, Cd, Np):
    """P, J_u, J_v of Eq. output_pred_vector (outputs stacked per step)."""
    q, n = Cd.shape
    P = np.zeros((q * Np, n))
    Ju = np.zeros((q * Np, Np))
    Jv = np.zeros((q * Np, Np))
    powers = [np.eye(n)]
    for _ in range(Np):
        powers.append(powers[-1] @ Ad)
    for i in range(1, Np + 1):
        P[q * (i - 1):q * i] = Cd @ powers[i]
        for j in range(1, i + 1):
            Ju[q * (i - 1):q * i, j - 1] = (Cd @ powers[i - j] @ Bd)[:, 0]
            Jv[q * (i - 1):q * i, j - 1] = (Cd @ powers[i - j] @ Fd)[:, 0]
    return P, Ju, Jv


def energy_weight(Np):
    """Q of Eq. J1: 0.5 Z^T Q Z = sum_{i < Np} u_i zd_i + u_Np zd_Np / 2."""
    M = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, 1.0, 0.0]])
    Q = np.zeros((3 * Np, 3 * Np))
    for i in range(Np):
        Q[3 * i:3 * i + 3, 3 * i:3 * i + 3] = M * (0.5 if i == Np - 1 else 1.0)
    return Q


def box_qp(H, f, lo, hi, x0=None, iters=100, tol=1e-12):
    """min 0.5 x^T H x + f^T x subject to lo <= x <= hi (H symmetric positive
    definite), by projected Newton: Newton steps on the variables not held at a
    bound by the gradient, an Armijo search along the projected path."""
    n = len(f)
    x = np.clip(np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64), lo, hi)
    obj = lambda y: 0.5 * y @ H @ y + f @ y
    for _ in range(iters):
        g = H @ x + f
        at_lo = (x <= lo) & (g > 0)
        at_hi = (x >= hi) & (g < 0)
        free = ~(at_lo | at_hi)
        d = np.zeros(n)
        if free.any():
            Hf = H[np.ix_(free, free)]
            d[free] = -np.linalg.solve(Hf, g[free])
        # projected gradient step on the bound variables (zero here) and the Newton step on the free ones
        fx = obj(x)
        t = 1.0
        while True:
            xn = np.clip(x + t * d, lo, hi)
            if obj(xn) <= fx + 1e-4 * g @ (xn - x) or t < 1e-12:
                break
            t *= 0.5
        done = np.max(np.abs(xn - x)) <= tol * (1.0 + np.max(np.abs(x)))
        x = xn
        if done:
            break
    return x


def qp_ineq(H, f, G, h, x0=None, tol=1e-11, iters=200):
    """min 0.5 x^T H x + f^T x subject to G x <= h (H symmetric positive
    definite), by a primal-dual interior-point method (Mehrotra's predictor-
    corrector on the slack form G x + s = h, s >= 0, with multipliers lam >= 0;
    each iteration solves the reduced Newton system (H + G^T diag(lam / s) G) dx
    = r), then polished on the active set the iterate identifies (the rows with
    s < lam): the equality-constrained KKT system solved exactly, kept if it is
    feasible with non-negative multipliers.  Returns x."""
    H = np.asarray(H, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n, m = len(f), len(h)
    if m == 0:
        return np.linalg.solve(H, -f)
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    s = np.maximum(h - G @ x, 1.0)
    lam = np.ones(m)
    scale = 1.0 + max(np.max(np.abs(f)), np.max(np.abs(h)))

    def step_to_boundary(v, dv):
        neg = dv < 0.0
        return min(1.0, float(np.min(-v[neg] / dv[neg]))) if neg.any() else 1.0

    for _ in range(iters):
        rd = H @ x + f + G.T @ lam  # dual residual
        rp = G @ x + s - h          # primal residual
        mu = float(lam @ s) / m
        if max(np.max(np.abs(rd)), np.max(np.abs(rp))) <= tol * scale and mu <= tol * scale:
            break

        def solve(rc):
            # H dx + G^T dlam = -rd, G dx + ds = -rp, lam ds + s dlam = rc:
            # eliminating ds and dlam gives (H + G^T W G) dx = -rd - G^T (rc / s + W rp)
            w = lam / s
            K = H + G.T @ (w[:, None] * G)
            dx = np.linalg.solve(K, -rd - G.T @ (rc / s + w * rp))
            ds = -rp - G @ dx
            dlam = (rc - lam * ds) / s
            return dx, ds, dlam

        # predictor (affine scaling), then the corrector with centring
        dx, ds, dlam = solve(-lam * s)
        a = min(step_to_boundary(s, ds), step_to_boundary(lam, dlam))
        mu_aff = float((lam + a * dlam) @ (s + a * ds)) / m
        sigma = (mu_aff / mu) ** 3 if mu > 0.0 else 0.0
        dx, ds, dlam = solve(-lam * s - ds * dlam + sigma * mu)
        a = 0.99 * min(step_to_boundary(s, ds), step_to_boundary(lam, dlam))
        x, s, lam = x + a * dx, s + a * ds, lam + a * dlam
    # polish: the active set's KKT system, exactly
    act = np.nonzero(s < lam)[0]
    k = len(act)
    if k <= n:
        GA = G[act]
        K = np.block([[H, GA.T], [GA, np.zeros((k, k))]])
        try:
            sol = np.linalg.solve(K, np.concatenate([-f, h[act]]))
        except np.linalg.LinAlgError:
            return x
        xp, la = sol[:n], sol[n:]
        eps = 1e-9 * scale
        if np.all(G @ xp <= h + eps) and np.all(la >= -eps):
            return xp
    return x


def ar_fit(x, order):
    """AR(p) coefficients a of x_t = sum_{i=1..p} a_i x_{t-i}, by least squares
    over every t of the record with p predecessors."""
    x = np.asarray(x, dtype=np.float64)
    if len(x) < 2 * order + 1:
        raise ValueError("AR fit: record shorter than 2 p + 1 samples")
    A = np.column_stack([x[order - i - 1:len(x) - i - 1] for i in range(order)])
    a, *_ = np.linalg.lstsq(A, x[order:], rcond=None)
    return a


def ar_predict(x, a, n):
    """The next n values of the record x under the AR model a (each
    prediction fed back as the newest sample)."""
    buf = list(np.asarray(x, dtype=np.float64)[-len(a):])
    out = []
    for _ in range(n):
        nxt = float(np.dot(a, buf[::-1]))
        out.append(nxt)
        buf = buf[1:] + [nxt]
    return np.asarray(out)


class ArForecaster:
    """Forecast of a signal sampled at the control rate: the last `window`
    samples fit an AR(order) model, run forward over the horizon."""

    def __init__(self, order, window):
        self.order, self.window = order, window
        self.hist = []

    def push(self, v):
        self.hist.append(float(v))
        if len(self.hist) > self.window:
            self.hist = self.hist[-self.window:]

    def ready(self):
        return len(self.hist) >= max(self.window, 2 * self.order + 1)

    def predict(self, n):
        a = ar_fit(self.hist, self.order)
        return ar_predict(self.hist, a, n)


class MPC:
    """Receding-horizon PTO force for the heaving body: one QP per control
    step dt_p, its first force applied with first-order hold.  z_lim, zd_lim:
    optional (min, max) bounds on the predicted displacement and velocity (Eq.
    path_constr); without them the QP is the force box alone."""

    def __init__(self, m_eff, k_h, c_r, dt_p, Np, lam1, lam2, f_max, z_lim=None, zd_lim=None):
        self.m, self.kh, self.dt_p, self.Np = m_eff, k_h, dt_p, Np
        self.lam1, self.lam2, self.f_max = lam1, lam2, f_max
        self.z_lim, self.zd_lim = z_lim, zd_lim
        A, B = continuous_model(m_eff, k_h, c_r)
        self.Ad, self.Bd, self.Fd, self.Cd = foh_model(A, B, dt_p)
        self.P, self.Ju, self.Jv = prediction_matrices(self.Ad, self.Bd, self.Fd, self.Cd, Np)
        Q = energy_weight(Np)
        D = np.eye(Np) - np.eye(Np, k=-1)  # du = D U - e1 u(k)
        self.D = D
        self.Hd = self.Ju.T @ Q @ self.Ju + 2.0 * lam1 * np.eye(Np)
        self.JuQ = self.Ju.T @ Q
        self.H = D.T @ self.Hd @ D + 2.0 * lam2 * np.eye(Np)
        self.H = 0.5 * (self.H + self.H.T)
        ev = np.linalg.eigvalsh(self.H)
        if ev[0] <= 0.0:
            raise ValueError(f"MPC Hessian not positive definite (min eigenvalue {ev[0]:.3e}); raise lam1 / lam2")
        self.U = None

    def solve(self, z, zd, F_now, F_exc_now, F_exc_future):
        """Optimal PTO forces over the horizon [N] from the state (z, zd), the
        force applied now and the excitation now and at the next Np control
        steps (F_exc_future, length Np)."""
        u_k = F_now / self.m
        v = np.concatenate([[F_exc_now], np.asarray(F_exc_future, dtype=np.float64)]) / self.m
        dv = np.diff(v)
        X = np.array([z, zd, u_k, v[0]])
        e1 = np.zeros(self.Np)
        e1[0] = 1.0
        f = self.D.T @ (self.Hd @ (-e1 * u_k) + self.JuQ @ (self.P @ X + self.Jv @ dv))
        umax = self.f_max / self.m
        x0 = None if self.U is None else np.concatenate([self.U[1:], self.U[-1:]])
        if self.z_lim is None and self.zd_lim is None:
            self.U = box_qp(self.H, f, -umax * np.ones(self.Np), umax * np.ones(self.Np), x0=x0)
        else:
            G, hv, ns = self.path_rows(X, u_k, dv, umax)
            # the state bounds softened by an exact penalty: one slack per bound
            # (the largest violation over the horizon), weighted far above any
            # multiplier the hard problem has, so the hard solution is returned
            # whenever one exists and the force limit always holds
            rho = 1e6 * (1.0 + np.max(np.abs(f)) + umax * np.max(np.abs(self.H)))
            Ha = np.zeros((self.Np + ns, self.Np + ns))
            Ha[:self.Np, :self.Np] = self.H
            Ha[self.Np:, self.Np:] = 1e-9 * np.max(np.abs(self.H)) * np.eye(ns)
            fa = np.concatenate([f, rho * np.ones(ns)])
            self.U = qp_ineq(Ha, fa, G, hv)[:self.Np]
        return self.U * self.m

    def path_rows(self, X, u_k, dv, umax):
        """G [U; e] <= h of Eq. path_constr: the predicted outputs Z = c + J_u D U
        with c = P X - J_u e_1 u(k) + J_v dv (Eq. output_pred_vector), their z
        and zd rows bounded up to one non-negative slack per bound e, and the
        force box.  Returns G, h and the number of slacks."""
        e1 = np.zeros(self.Np)
        e1[0] = 1.0
        c = self.P @ X - self.Ju @ (e1 * u_k) + self.Jv @ dv
        M = self.Ju @ self.D
        blocks, rhs = [], []
        for off, lim in ((0, self.z_lim), (1, self.zd_lim)):
            if lim is None:
                continue
            lo, hi = lim
            Mi, ci = M[off::3], c[off::3]
            blocks += [(Mi, hi - ci), (-Mi, -(lo - ci))]
        ns = len(blocks)
        rows = [np.hstack([np.eye(self.Np), np.zeros((self.Np, ns))]),
                np.hstack([-np.eye(self.Np), np.zeros((self.Np, ns))])]
        rhs = [umax * np.ones(self.Np), umax * np.ones(self.Np)]
        for q, (Mi, r) in enumerate(blocks):
            S = np.zeros((self.Np, ns))
            S[:, q] = -1.0
            rows.append(np.hstack([Mi, S]))
            rhs.append(r)
        rows.append(np.hstack([np.zeros((ns, self.Np)), -np.eye(ns)]))
        rhs.append(np.zeros(ns))
        return np.vstack(rows), np.concatenate(rhs), ns

    def predicted(self, z, zd, F_now, F_exc_now, F_exc_future, U=None):
        """The predicted outputs [z, zd, u] over the horizon (rows per step)
        for the force sequence U (default: the last solution), in SI units."""
        u_k = F_now / self.m
        v = np.concatenate([[F_exc_now], np.asarray(F_exc_future, dtype=np.float64)]) / self.m
        X = np.array([z, zd, u_k, v[0]])
        e1 = np.zeros(self.Np)
        e1[0] = 1.0
        Uu = self.U if U is None else np.asarray(U, dtype=np.float64) / self.m
        Z = self.P @ X + self.Ju @ (self.D @ Uu - e1 * u_k) + self.Jv @ np.diff(v)
        out = Z.reshape(self.Np, 3).copy()
        out[:, 2] *= self.m
        return out

    def ramp(self, F_now, F_next, nsub):
        """First-order hold of the force over one control step split into nsub
        solver steps: the force at the start of each solver step."""
        s = np.arange(nsub) / nsub
        return F_now + s * (F_next - F_now)


def hydrostatic_stiffness(rho_w, g, width):
    """k_h = rho_w g W (per unit span) of a box with vertical sides."""
    return rho_w * g * width


def identify_free_decay(t, z, k_h):
    """Effective mass and linear damping from a free-decay record z(t) about
    its equilibrium: the damped period from successive zero crossings, the
    damping ratio from the logarithmic decrement of successive peaks,
    w_n = w_d / sqrt(1 - zeta^2), m_eff = k_h / w_n^2, c_r = 2 zeta w_n m_eff."""
    t = np.asarray(t, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    zc = [t[i] - z[i] * (t[i + 1] - t[i]) / (z[i + 1] - z[i]) for i in range(len(z) - 1) if z[i] * z[i + 1] < 0]
    if len(zc) < 3:
        raise ValueError("free decay: fewer than three zero crossings")
    Td = 2.0 * np.mean(np.diff(zc))
    peaks = []
    for a, b in zip(zc[:-1], zc[1:]):
        sel = (t > a) & (t < b)
        if sel.any():
            peaks.append(np.max(np.abs(z[sel])))
    if len(peaks) < 2:
        raise ValueError("free decay: fewer than two peaks")
    delta = np.mean(np.log(np.asarray(peaks[:-1]) / np.asarray(peaks[1:]))) * 2.0  # per full period
    zeta = delta / math.sqrt(4.0 * math.pi ** 2 + delta ** 2)
    wd = 2.0 * math.pi / Td
    wn = wd / math.sqrt(1.0 - zeta ** 2)
    m_eff = k_h / wn ** 2
    return m_eff, 2.0 * zeta * wn * m_eff, wn, zeta
