"""Exact log-likelihood and gradient of the linear-Gaussian model (test infrastructure only).

For the LG-diag family (theta = (a[dx], log q[dx], log r[dy]);
x_0 ~ N(0, I), x_t = diag(a) x_{t-1} + diag(q) v_t, y_t = H x_t + diag(r) w_t)
the Bayesian filtering recursion of Sec. II (Eqs. Chapman-Kolmogrov and
filtering_bayes_) has the closed form of the Kalman filter.  Its likelihood
p(y_{1:T}|theta) is what the particle filter's estimate (Eq. likelihood_pf_)
is unbiased for, so it pins the particle filter; the gradient is carried by a
forward-mode tangent recursion through the same filter.

``joint_loglik`` is an independent brute-force check: the density of the
stacked vector y_{1:T} under its full joint Gaussian law.
"""
import numpy as np

LOG_2PI = np.log(2.0 * np.pi)


def _unpack(theta, dx, dy):
    theta = np.asarray(theta, dtype=np.float64)
    a = theta[:dx]
    q = np.exp(theta[dx:2 * dx])
    r = np.exp(theta[2 * dx:2 * dx + dy])
    return a, q, r


def loglik_grad(theta, y, H=None, dx=1, dy=1):
    """Kalman-filter log p(y_{1:T}|theta) and its gradient w.r.t. theta (FP64)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, dy)
    T = y.shape[0]
    H = np.eye(dy, dx) if H is None else np.asarray(H, dtype=np.float64).reshape(dy, dx)
    a, q, r = _unpack(theta, dx, dy)
    D = 2 * dx + dy
    A = np.diag(a)
    Q = np.diag(q * q)
    R = np.diag(r * r)
    # parameter derivatives of A, Q, R
    dA = np.zeros((D, dx, dx))
    dQ = np.zeros((D, dx, dx))
    dR = np.zeros((D, dy, dy))
    for k in range(dx):
        dA[k, k, k] = 1.0
        dQ[dx + k, k, k] = 2.0 * q[k] * q[k]          # d(q^2)/dlog q
    for m in range(dy):
        dR[2 * dx + m, m, m] = 2.0 * r[m] * r[m]      # d(r^2)/dlog r
    m_ = np.zeros(dx)
    P = np.eye(dx)
    dm = np.zeros((D, dx))
    dP = np.zeros((D, dx, dx))
    ll = 0.0
    g = np.zeros(D)
    for t in range(T):
        # predict
        mp = A @ m_
        Pp = A @ P @ A.T + Q
        dmp = np.einsum("dij,j->di", dA, m_) + dm @ A.T
        dPp = (np.einsum("dij,jk,lk->dil", dA, P, A) + np.einsum("ij,djk,lk->dil", A, dP, A)
               + np.einsum("ij,jk,dlk->dil", A, P, dA) + dQ)
        # update
        S = H @ Pp @ H.T + R
        Si = np.linalg.inv(S)
        e = y[t] - H @ mp
        sign, logdet = np.linalg.slogdet(S)
        ll += -0.5 * (e @ Si @ e + logdet + dy * LOG_2PI)
        dS = np.einsum("ij,djk,lk->dil", H, dPp, H) + dR
        de = -dmp @ H.T
        Sie = Si @ e
        for d in range(D):
            g[d] += -0.5 * (2.0 * Sie @ de[d] - Sie @ dS[d] @ Sie + np.trace(Si @ dS[d]))
        K = Pp @ H.T @ Si
        dK = np.einsum("dij,kj->dik", dPp, H) @ Si - np.einsum("ij,kj,kl,dlm,mn->din", Pp, H, Si, dS, Si)
        m_ = mp + K @ e
        P = Pp - K @ H @ Pp
        dm = dmp + np.einsum("dij,j->di", dK, e) + de @ K.T
        dP = dPp - np.einsum("dij,jk,kl->dil", dK, H, Pp) - np.einsum("ij,jk,dkl->dil", K, H, dPp)
    return ll, g


def joint_loglik(theta, y, H=None, dx=1, dy=1):
    """log N(vec(y_{1:T}); 0, Sigma) with Sigma built from the model's covariances (small T)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, dy)
    T = y.shape[0]
    H = np.eye(dy, dx) if H is None else np.asarray(H, dtype=np.float64).reshape(dy, dx)
    a, q, r = _unpack(theta, dx, dy)
    A = np.diag(a)
    Q = np.diag(q * q)
    # state covariances Cov(x_s, x_t) for s, t in 1..T
    Vx = [None] * (T + 1)
    Vx[0] = np.eye(dx)
    for t in range(1, T + 1):
        Vx[t] = A @ Vx[t - 1] @ A.T + Q
    Sig = np.zeros((T * dy, T * dy))
    for s in range(1, T + 1):
        for t in range(s, T + 1):
            C = np.linalg.matrix_power(A, t - s) @ Vx[s]        # Cov(x_t, x_s)
            blk = H @ C @ H.T
            Sig[(t - 1) * dy:t * dy, (s - 1) * dy:s * dy] = blk
            Sig[(s - 1) * dy:s * dy, (t - 1) * dy:t * dy] = blk.T
    Sig += np.kron(np.eye(T), np.diag(r * r))
    v = y.reshape(-1)
    sign, logdet = np.linalg.slogdet(Sig)
    return float(-0.5 * (v @ np.linalg.solve(Sig, v) + logdet + T * dy * LOG_2PI))
