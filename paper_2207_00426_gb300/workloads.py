"""Seeded synthetic workloads shaped like the paper's tracking experiments.

This module only draws random inputs and simulates the state-space models;
it contains none of the smoother's arithmetic.  Both the CUDA path (tests,
bench) and the FP64 oracle read the arrays it returns.

Workloads
---------
linear_cv       2-D constant-velocity model, n_x = 4, n_y = 2 (positions
                observed), dt = 0.1, q = 0.1, sigma = 0.5, x0 ~ N(0, I),
                m0 = 0, P0 = I.
random_lgssm    random time-varying linear-Gaussian model (for tests).
ct_sequence     coordinated-turn bearings-only tracking (Sec. 6.2 of the
                paper): x = (p_x, p_y, v_x, v_y, omega), dt = 0.01,
                q_c = 0.01, q_omega = 0.1, bearings from sensors (-1.5, 0.5)
                and (1, 1) with sigma = 0.05 rad.  x0: p = 0, speed
                U(0.5, 2), heading U(0, 2 pi), omega N(0, 0.3^2); prior
                m0 = x0, P0 = 0.1^2 I.
ct_batch        many independent CT sequences of lengths U{lo..hi},
                concatenated, with int64 offsets.
All arrays are float64 NumPy; callers cast.
"""
import numpy as np

CT_SENSORS = np.array([[-1.5, 0.5], [1.0, 1.0]])
CT_THETA_TRUE = np.log(np.array([0.05, 0.01, 0.1]))   # (sigma, q_c, q_omega)
CT_DT = 0.01


def _cv_matrices(dt, q, sigma):
    I2, Z2 = np.eye(2), np.zeros((2, 2))
    F = np.block([[I2, dt * I2], [Z2, I2]])
    SQ = np.sqrt(q) * np.block([[np.sqrt(dt ** 3 / 3) * I2, Z2],
                                [np.sqrt(3 * dt) / 2 * I2, np.sqrt(dt) / 2 * I2]])
    H = np.hstack([I2, Z2])
    SR = sigma * I2
    return F, SQ, H, SR


def linear_cv(n=1000, seed=0, dt=0.1, q=0.1, sigma=0.5):
    rng = np.random.default_rng(seed)
    F, SQ, H, SR = _cv_matrices(dt, q, sigma)
    nx, ny = 4, 2
    x = np.zeros((n + 1, nx))
    x[0] = rng.standard_normal(nx)
    y = np.zeros((n, ny))
    for t in range(n):
        x[t + 1] = F @ x[t] + SQ @ rng.standard_normal(nx)
        y[t] = H @ x[t + 1] + SR @ rng.standard_normal(ny)
    return dict(F=np.tile(F, (n, 1, 1)), c=np.zeros((n, nx)),
                SQ=np.tile(SQ, (n, 1, 1)), H=np.tile(H, (n, 1, 1)),
                d=np.zeros((n, ny)), SR=np.tile(SR, (n, 1, 1)),
                y=y, m0=np.zeros(nx), N0=np.eye(nx), x=x)


def _rand_lower(rng, k, scale):
    L = np.tril(rng.standard_normal((k, k))) * scale
    L[np.diag_indices(k)] = np.abs(L[np.diag_indices(k)]) + scale
    return L


def random_lgssm(n, nx, ny, seed=0, scale=0.3):
    """Random time-varying linear-Gaussian model and a simulated path."""
    rng = np.random.default_rng(seed)
    F = np.stack([np.eye(nx) + scale * rng.standard_normal((nx, nx)) / np.sqrt(nx)
                  for _ in range(n)])
    # keep every transition contractive so long sequences stay bounded
    F *= np.minimum(1.0, 0.98 / np.linalg.norm(F, ord=2, axis=(1, 2)))[:, None, None]
    c = 0.1 * rng.standard_normal((n, nx))
    SQ = np.stack([_rand_lower(rng, nx, scale) for _ in range(n)])
    H = rng.standard_normal((n, ny, nx))
    d = 0.1 * rng.standard_normal((n, ny))
    SR = np.stack([_rand_lower(rng, ny, scale) for _ in range(n)])
    m0 = rng.standard_normal(nx)
    N0 = _rand_lower(rng, nx, 1.0)
    x = np.zeros((n + 1, nx))
    x[0] = m0 + N0 @ rng.standard_normal(nx)
    y = np.zeros((n, ny))
    for t in range(n):
        x[t + 1] = F[t] @ x[t] + c[t] + SQ[t] @ rng.standard_normal(nx)
        y[t] = H[t] @ x[t + 1] + d[t] + SR[t] @ rng.standard_normal(ny)
    return dict(F=F, c=c, SQ=SQ, H=H, d=d, SR=SR, y=y, m0=m0, N0=N0, x=x)


def _ct_step(x, dt):
    px, py, vx, vy, w = x
    a = w * dt
    if abs(a) < 1e-9:
        S, C = dt, 0.5 * w * dt * dt
    else:
        S, C = np.sin(a) / w, (1.0 - np.cos(a)) / w
    ca, sa = np.cos(a), np.sin(a)
    return np.array([px + S * vx - C * vy, py + C * vx + S * vy,
                     ca * vx - sa * vy, sa * vx + ca * vy, w])


def _ct_noise_factor(dt, qc, qw):
    L = np.zeros((5, 5))
    for i in (0, 1):
        L[i, i] = np.sqrt(qc * dt ** 3 / 3.0)
        L[i + 2, i] = np.sqrt(qc * 3.0 * dt) / 2.0
        L[i + 2, i + 2] = np.sqrt(qc * dt) / 2.0
    L[4, 4] = np.sqrt(qw * dt)
    return L


def _simulate_ct(rng, n, dt, sigma, qc, qw, sensors):
    speed = rng.uniform(0.5, 2.0)
    heading = rng.uniform(0.0, 2.0 * np.pi)
    w0 = 0.3 * rng.standard_normal()
    x0 = np.array([0.0, 0.0, speed * np.cos(heading), speed * np.sin(heading), w0])
    L = _ct_noise_factor(dt, qc, qw)
    x = np.zeros((n + 1, 5))
    x[0] = x0
    y = np.zeros((n, 2))
    for t in range(n):
        x[t + 1] = _ct_step(x[t], dt) + L @ rng.standard_normal(5)
        b = np.arctan2(x[t + 1, 1] - sensors[:, 1], x[t + 1, 0] - sensors[:, 0])
        b = b + sigma * rng.standard_normal(2)
        y[t] = b - 2.0 * np.pi * np.floor(b / (2.0 * np.pi) + 0.5)
    return x, y


def ct_sequence(n=10_000, seed=1, dt=CT_DT, theta=CT_THETA_TRUE,
                sensors=CT_SENSORS, prior_std=0.1):
    rng = np.random.default_rng(seed)
    sigma, qc, qw = np.exp(theta)
    x, y = _simulate_ct(rng, n, dt, sigma, qc, qw, sensors)
    return dict(y=y, x=x, m0=x[0].copy(), N0=prior_std * np.eye(5),
                theta=np.array(theta, dtype=np.float64), dt=dt,
                sensors=np.array(sensors, dtype=np.float64))


def ct_batch(batch=4096, lo=100, hi=5000, seed=3, dt=CT_DT, theta=CT_THETA_TRUE,
             sensors=CT_SENSORS, prior_std=0.1, lengths=None):
    """Independent CT sequences; y rows of sequence b are
    y[offsets[b]:offsets[b+1]], its prior m0[b], N0[b].  All sequences are
    simulated together (vectorised over the batch)."""
    rng = np.random.default_rng(seed)
    sigma, qc, qw = np.exp(theta)
    if lengths is None:
        lengths = rng.integers(lo, hi + 1, size=batch)
    lengths = np.asarray(lengths, dtype=np.int64)
    B = len(lengths)
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    speed = rng.uniform(0.5, 2.0, B)
    heading = rng.uniform(0.0, 2.0 * np.pi, B)
    w0 = 0.3 * rng.standard_normal(B)
    x = np.stack([np.zeros(B), np.zeros(B), speed * np.cos(heading), speed * np.sin(heading), w0], 1)
    m0 = x.copy()
    L = _ct_noise_factor(dt, qc, qw)
    nmax = int(lengths.max())
    y = np.zeros((int(offsets[-1]), 2))
    for t in range(nmax):
        px, py, vx, vy, w = x.T
        a = w * dt
        small = np.abs(a) < 1e-9
        wsafe = np.where(small, 1.0, w)
        S = np.where(small, dt, np.sin(a) / wsafe)
        C = np.where(small, 0.5 * w * dt * dt, (1.0 - np.cos(a)) / wsafe)
        ca, sa = np.cos(a), np.sin(a)
        x = np.stack([px + S * vx - C * vy, py + C * vx + S * vy,
                      ca * vx - sa * vy, sa * vx + ca * vy, w], 1)
        x = x + rng.standard_normal((B, 5)) @ L.T
        bear = np.arctan2(x[:, 1:2] - sensors[None, :, 1], x[:, 0:1] - sensors[None, :, 0])
        bear = bear + sigma * rng.standard_normal((B, 2))
        bear = bear - 2.0 * np.pi * np.floor(bear / (2.0 * np.pi) + 0.5)
        live = t < lengths
        rows = offsets[:-1][live] + t
        y[rows] = bear[live]
    N0 = np.tile(prior_std * np.eye(5), (B, 1, 1))
    return dict(y=y, offsets=offsets, m0=m0, N0=N0,
                theta=np.array(theta, dtype=np.float64), dt=dt,
                sensors=np.array(sensors, dtype=np.float64))


# Stochastic Ricker population model with Poisson counts: a = 44.7, b = 10,
# Q = 0.3^2, known initial state x_0 = log 7.
RICKER_THETA_TRUE = np.log(np.array([44.7, 10.0, 0.09]))   # (a, b, Q)
RICKER_X0 = float(np.log(7.0))


def ricker_batch(lengths, seed=0, theta=RICKER_THETA_TRUE, x0=RICKER_X0):
    """Independent Ricker sequences (vectorised over the batch):
    x_k = log a + x_{k-1} - exp(x_{k-1}) + q_k, y_k ~ Poisson(b exp(x_k)),
    x_0 = x0.  Returns y [sum n, 1], offsets, x (states, state layout),
    m0 [B, 1] = x0, N0 [B, 1, 1] = 0 (a point mass), theta."""
    rng = np.random.default_rng(seed)
    a, b, q = np.exp(theta)
    lengths = np.asarray(lengths, dtype=np.int64)
    B = len(lengths)
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    x = np.full(B, x0)
    xs = np.zeros((int(offsets[-1]) + B, 1))
    y = np.zeros((int(offsets[-1]), 1))
    for bb in range(B):
        xs[offsets[bb] + bb, 0] = x0
    for t in range(int(lengths.max())):
        x = np.log(a) + x - np.exp(x) + np.sqrt(q) * rng.standard_normal(B)
        counts = rng.poisson(b * np.exp(x))
        for bb in range(B):
            if t < lengths[bb]:
                y[offsets[bb] + t, 0] = counts[bb]
                xs[offsets[bb] + bb + t + 1, 0] = x[bb]
    return {"y": y, "offsets": offsets, "x": xs, "m0": np.full((B, 1), x0),
            "N0": np.zeros((B, 1, 1)), "theta": np.asarray(theta, dtype=np.float64)}

