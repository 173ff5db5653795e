"""State-space models of the experiments (Sec. 6).  Oracle: test
infrastructure only.

Coordinated-turn (CT) bearings-only model (Sec. 6.2).  The paper follows
Arasaratnam & Haykin's parameterisation without printing it; the readings
taken here are:
* state x = (p_x, p_y, v_x, v_y, omega), time step dt;
* dynamics (exact discretisation of a constant turn):
    p' = p + [[S, -C], [C, S]] v,  v' = [[cos a, -sin a], [sin a, cos a]] v,
    omega' = omega,   a = omega dt,  S = sin(a)/omega,  C = (1 - cos a)/omega,
  with C evaluated as 2 sin^2(a/2)/omega (same value, no cancellation) and,
  for |a| < 1e-3, the series S = dt (1 - a^2/6 + a^4/120),
  C = dt (a/2 - a^3/24 + a^5/720);
* additive process noise with covariance
    q_c [[dt^3/3 I2, dt^2/2 I2], [dt^2/2 I2, dt I2]] on (p, v) and q_w dt on
  omega, whose lower Cholesky factor is written in closed form;
* bearings h_i(x) = atan2(p_y - s_y^i, p_x - s_x^i) from sensors
  (-1.5, 0.5) and (1, 1), noise sigma^2 I2;
* parameters theta = (log sigma, log q_c, log q_w), or, with one noise
  level per sensor as in the sqrt(R_11) estimation of Sec. 6.4,
  theta = (log sqrt(R_11), log q_c, log q_w, log sqrt(R_22)) and noise
  diag(R_11, R_22).
"""
import numpy as np

SENSORS = np.array([[-1.5, 0.5], [1.0, 1.0]])


def wrap_angle(a):
    """Wrap to [-pi, pi): a - 2 pi floor(a / (2 pi) + 1/2)."""
    return a - 2.0 * np.pi * np.floor(a / (2.0 * np.pi) + 0.5)


def _turn_coeffs(w, dt):
    """S = sin(w dt)/w and C = (1 - cos(w dt))/w with the small-angle series."""
    a = w * dt
    if abs(a) < 1e-3:
        S = dt * (1.0 - a * a / 6.0 + a ** 4 / 120.0)
        C = dt * (a / 2.0 - a ** 3 / 24.0 + a ** 5 / 720.0)
    else:
        S = np.sin(a) / w
        C = 2.0 * np.sin(0.5 * a) ** 2 / w
    return S, C


def _turn_coeff_derivs(w, dt):
    """dS/dw and dC/dw; series in a = w dt for |a| < 0.1 (terms to a^8),
    closed form (a cos a - sin a)/a^2 and (a sin a - (1 - cos a))/a^2 times
    dt^2 otherwise."""
    a = w * dt
    if abs(a) < 0.1:
        dsa = -a / 3.0 + a ** 3 / 30.0 - a ** 5 / 840.0 + a ** 7 / 45360.0
        dca = 0.5 - a * a / 8.0 + a ** 4 / 144.0 - a ** 6 / 5760.0 + a ** 8 / 403200.0
    else:
        dsa = (a * np.cos(a) - np.sin(a)) / (a * a)
        dca = (a * np.sin(a) - 2.0 * np.sin(0.5 * a) ** 2) / (a * a)
    return dt * dt * dsa, dt * dt * dca


class CTBearings:
    """Coordinated-turn bearings-only model with parameters theta."""
    nx = 5
    ny = 2

    def __init__(self, theta, dt=0.01, sensors=SENSORS):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.dt = float(dt)
        self.sensors = np.asarray(sensors, dtype=np.float64)
        if self.theta.size not in (3, 4):
            raise ValueError("theta has 3 or 4 entries")
        self.sigma = np.exp(self.theta[0])
        self.sigma2 = np.exp(self.theta[3]) if self.theta.size == 4 else self.sigma
        self.qc = np.exp(self.theta[1])
        self.qw = np.exp(self.theta[2])

    # transition ------------------------------------------------------------
    def f(self, x):
        px, py, vx, vy, w = x
        S, C = _turn_coeffs(w, self.dt)
        a = w * self.dt
        ca, sa = np.cos(a), np.sin(a)
        return np.array([px + S * vx - C * vy,
                         py + C * vx + S * vy,
                         ca * vx - sa * vy,
                         sa * vx + ca * vy,
                         w])

    def jac_f(self, x):
        px, py, vx, vy, w = x
        dt = self.dt
        S, C = _turn_coeffs(w, dt)
        dS, dC = _turn_coeff_derivs(w, dt)
        a = w * dt
        ca, sa = np.cos(a), np.sin(a)
        return np.array([
            [1.0, 0.0, S, -C, vx * dS - vy * dC],
            [0.0, 1.0, C, S, vx * dC + vy * dS],
            [0.0, 0.0, ca, -sa, -dt * sa * vx - dt * ca * vy],
            [0.0, 0.0, sa, ca, dt * ca * vx - dt * sa * vy],
            [0.0, 0.0, 0.0, 0.0, 1.0]])

    def Q(self):
        dt, qc, qw = self.dt, self.qc, self.qw
        Q = np.zeros((5, 5))
        for i in (0, 1):
            Q[i, i] = qc * dt ** 3 / 3.0
            Q[i, i + 2] = Q[i + 2, i] = qc * dt ** 2 / 2.0
            Q[i + 2, i + 2] = qc * dt
        Q[4, 4] = qw * dt
        return Q

    def SQ(self):
        """Closed-form lower Cholesky factor of Q (per axis
        sqrt(q_c) [[sqrt(dt^3/3), 0], [sqrt(3 dt)/2, sqrt(dt)/2]])."""
        dt, qc, qw = self.dt, self.qc, self.qw
        L = np.zeros((5, 5))
        for i in (0, 1):
            L[i, i] = np.sqrt(qc * dt ** 3 / 3.0)
            L[i + 2, i] = np.sqrt(qc) * np.sqrt(3.0 * dt) / 2.0
            L[i + 2, i + 2] = np.sqrt(qc) * np.sqrt(dt) / 2.0
        L[4, 4] = np.sqrt(qw * dt)
        return L

    # observation -----------------------------------------------------------
    def h(self, x):
        return np.arctan2(x[1] - self.sensors[:, 1], x[0] - self.sensors[:, 0])

    def jac_h(self, x):
        dx = x[0] - self.sensors[:, 0]
        dy = x[1] - self.sensors[:, 1]
        r2 = dx * dx + dy * dy
        J = np.zeros((2, 5))
        J[:, 0] = -dy / r2
        J[:, 1] = dx / r2
        return J

    def branch(self, z, ref):
        """Bearings are angles: take the branch of z nearest to ref."""
        return ref + wrap_angle(z - ref)

    def SR(self):
        return np.diag([self.sigma, self.sigma2])

    # parameter derivatives (forward-mode gradient) ---------------------------
    def dSQ_dtheta(self):
        """d SQ / d theta_j, trailing axis j: SQ scales with sqrt(q_c) on the
        (p, v) block and with sqrt(q_omega) on omega, so the derivatives in
        log q_c and log q_omega are half of those parts; sigma does not
        enter."""
        L = self.SQ()
        D = np.zeros((5, 5, self.theta.size))
        D[:4, :4, 1] = 0.5 * L[:4, :4]
        D[4, 4, 2] = 0.5 * L[4, 4]
        return D

    def dSR_dtheta(self):
        """d SR / d theta_j: SR = diag(sigma, sigma_2) with sigma = e^theta_0
        (and sigma_2 = e^theta_3 when theta has four entries, else sigma)."""
        D = np.zeros((2, 2, self.theta.size))
        if self.theta.size == 4:
            D[0, 0, 0] = self.sigma
            D[1, 1, 3] = self.sigma2
        else:
            D[:, :, 0] = self.SR()
        return D


class LinearCV:
    """Linear constant-velocity model of the 2-D tracking example:
    x = (p_x, p_y, v_x, v_y), F = [[I, dt I], [0, I]], white-noise
    acceleration Q = q [[dt^3/3 I, dt^2/2 I], [dt^2/2 I, dt I]],
    H = [I 0], R = sigma^2 I."""
    nx = 4
    ny = 2

    def __init__(self, dt=0.1, q=0.1, sigma=0.5):
        self.dt, self.q, self.sigma = float(dt), float(q), float(sigma)

    def matrices(self):
        dt, q = self.dt, self.q
        I2 = np.eye(2)
        Z2 = np.zeros((2, 2))
        F = np.block([[I2, dt * I2], [Z2, I2]])
        Q = q * np.block([[dt ** 3 / 3 * I2, dt ** 2 / 2 * I2],
                          [dt ** 2 / 2 * I2, dt * I2]])
        SQ = np.sqrt(q) * np.block([[np.sqrt(dt ** 3 / 3) * I2, Z2],
                                    [np.sqrt(3 * dt) / 2 * I2, np.sqrt(dt) / 2 * I2]])
        H = np.hstack([I2, Z2])
        R = self.sigma ** 2 * I2
        SR = self.sigma * I2
        return F, Q, SQ, H, R, SR


class RickerPoisson:
    """Stochastic Ricker population model with Poisson counts (Sec. 6.1):
        x_k = log a + x_{k-1} - exp(x_{k-1}) + q_k,  q_k ~ N(0, Q),
        y_k | x_k ~ Poisson(b exp(x_k)),  x_0 = log c (a point mass).
    The observation noise is not additive: its conditional mean and variance
    are both b exp(x), so the SLR takes the per-point conditional factor
    sqrt(b exp(X_i)) (Sec. 4.3, general GSLR).  Parameters theta =
    (log a, log b, log Q); the paper's values a = 44.7, b = 10, Q = 0.3^2,
    c = 7."""
    nx = 1
    ny = 1

    def __init__(self, theta):
        self.a, self.b, self.q = (float(np.exp(t)) for t in theta)

    def f(self, x):
        return np.log(self.a) + x - np.exp(x)

    def jac_f(self, x):
        return np.array([[1.0 - np.exp(x[0])]])

    def SQ(self):
        return np.array([[np.sqrt(self.q)]])

    def h(self, x):
        """Conditional mean E[y | x]."""
        return self.b * np.exp(x)

    def jac_h(self, x):
        return np.array([[self.b * np.exp(x[0])]])

    def cond_SR(self, x):
        """Lower factor of the conditional covariance Var[y | x]."""
        return np.array([[np.sqrt(self.b * np.exp(x[0]))]])

    def SR(self):
        raise TypeError("the observation noise of this model depends on the state: use cond_SR")

    def branch(self, z, ref):
        return z

