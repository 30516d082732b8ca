"""Seeded synthetic workloads (input generators only).

This module holds no arithmetic of the particle filter or of the sampler: it
draws model matrices, true parameters and observation series y_{1:T} with
numpy's PCG64 generator, by simulating the state-space model of Sec. II
(Eqs. xt, yt) forward once, in FP64, and storing y as FP32.  Both the CUDA
path and the CPU oracle consume what it returns.

Workloads (data seed 12345 + index):
  lg1     1-D linear-Gaussian, theta = (a, log sigma_v, log sigma_w), D=3,
          theta* = (0.8, log 0.5, log 1.0), T=100, N=64, M=128, K=10 Langevin.
  lg4     LG-diag d_x=4, d_y=2, a* ~ U(0, 0.95), H (2x4) ~ N(0,1)/sqrt(4),
          theta = (a[4], log q[4], log r[2]), D=10, q*=0.5, r*=1.0,
          T=250, N=1024, M=1024.
  sv      stochastic volatility, theta = (mu, atanh phi, log sigma), D=3,
          theta* = (-1, atanh 0.95, log 0.25), T=500, N=4096, M=2048, K=20.
  lg16    LG-diag d_x=d_y=16, H=I, D=48, a* ~ U(0, 0.95), q*=0.5, r*=1.0,
          T=200, N=2048, M=1024, K=30, prior N((0.5, log 0.5, 0), (0.15, 0.3, 0.3)^2)
          per dimension (the others use N(0, I)).
  lgssm   the linear-Gaussian model of Sec. IV-A with the optimal proposal,
          theta = (mu, phi, sigma), theta* = (0.75, 1, 1), uniform priors, T=500,
          N=64, M=250, K=15.
Step sizes: Langevin 0.085*sqrt(500/T), random walk 0.175*sqrt(500/T), scaled
from the values the paper tuned for its T=500 linear-Gaussian model; the 48-parameter
lg16 uses 0.03*sqrt(200/T) (random walk 0.06*sqrt(200/T)).
"""
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

LG_DIAG = 0
SV = 1
LG_OPT = 2
GAUSSIAN_PRIOR = 0
UNIFORM_PRIOR = 1


@dataclass
class Workload:
    name: str
    family: int
    dx: int
    dy: int
    D: int
    T: int
    N: int
    M: int
    K: int
    theta_star: np.ndarray
    y: np.ndarray                       # (T, dy) float32
    H: Optional[np.ndarray] = None      # (dy, dx) float32 or None (identity)
    proposal: str = "langevin"
    gamma: float = 0.1
    seed: int = 777
    data_seed: int = 12345
    prior_mean: Optional[np.ndarray] = None   # None: N(0, I) prior on theta
    prior_std: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)
    prior_kind: int = GAUSSIAN_PRIOR          # UNIFORM_PRIOR: U(prior_mean[d], prior_std[d])
    hmc_steps: int = 1                        # leapfrog steps of the "hmc" proposal
    nuts_depth: int = 3                       # maximum doublings of the "nuts" proposal
    nuts_weight: int = 0                      # 0: the NUTS kernel's reversal, 1: momentum reversal

    @property
    def particle_steps(self) -> int:
        return self.N * self.M * self.T

    def with_sizes(self, **kw) -> "Workload":
        """Same model and data, other sizes (T may only shrink: y is truncated)."""
        w = replace(self, **kw)
        if "T" in kw:
            if kw["T"] > self.y.shape[0]:
                raise ValueError("T larger than the simulated series")
            w.y = np.ascontiguousarray(self.y[:kw["T"]])
        return w


def step_sizes(T: int):
    s = np.sqrt(500.0 / T)
    # an HMC move takes Langevin-sized leapfrog steps (one step is the Langevin move)
    return {"langevin": 0.085 * s, "rw": 0.175 * s, "hmc": 0.085 * s, "nuts": 0.085 * s}


def simulate_lg(rng, a, q, r, H, T):
    """Simulate x_0 ~ N(0,I), x_t = a*x_{t-1} + q*v_t, y_t = H x_t + r*w_t (FP64)."""
    dx = a.shape[0]
    dy = r.shape[0]
    Hm = np.eye(dy, dx) if H is None else H.astype(np.float64)
    x = rng.standard_normal(dx)
    ys = np.zeros((T, dy))
    for t in range(T):
        x = a * x + q * rng.standard_normal(dx)
        ys[t] = Hm @ x + r * rng.standard_normal(dy)
    return ys.astype(np.float32)


def simulate_sv(rng, mu, phi, sig, T):
    x = mu + sig / np.sqrt(1.0 - phi * phi) * rng.standard_normal()
    ys = np.zeros((T, 1))
    for t in range(T):
        x = mu + phi * (x - mu) + sig * rng.standard_normal()
        ys[t, 0] = np.exp(0.5 * x) * rng.standard_normal()
    return ys.astype(np.float32)


def lg1(T=100, N=64, M=128, K=10, proposal="langevin") -> Workload:
    seed = 12345 + 0
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.array([0.8, np.log(0.5), np.log(1.0)])
    y = simulate_lg(rng, th[:1], np.exp(th[1:2]), np.exp(th[2:3]), None, T)
    return Workload("lg1", LG_DIAG, 1, 1, 3, T, N, M, K, th, y, None, proposal,
                    step_sizes(T)[proposal], 777, seed)


def lg4(T=250, N=1024, M=1024, K=10, proposal="langevin") -> Workload:
    seed = 12345 + 1
    rng = np.random.Generator(np.random.PCG64(seed))
    dx, dy = 4, 2
    a = rng.uniform(0.0, 0.95, size=dx)
    H = (rng.standard_normal((dy, dx)) / np.sqrt(dx)).astype(np.float32)
    th = np.concatenate([a, np.full(dx, np.log(0.5)), np.full(dy, np.log(1.0))])
    y = simulate_lg(rng, a, np.full(dx, 0.5), np.full(dy, 1.0), H, T)
    return Workload("lg4", LG_DIAG, dx, dy, 2 * dx + dy, T, N, M, K, th, y, H, proposal,
                    step_sizes(T)[proposal], 778, seed)


def sv(T=500, N=4096, M=2048, K=20, proposal="langevin") -> Workload:
    seed = 12345 + 2
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.array([-1.0, np.arctanh(0.95), np.log(0.25)])
    y = simulate_sv(rng, th[0], np.tanh(th[1]), np.exp(th[2]), T)
    return Workload("sv", SV, 1, 1, 3, T, N, M, K, th, y, None, proposal,
                    step_sizes(T)[proposal], 779, seed)


def lg16(T=200, N=2048, M=1024, K=30, proposal="langevin") -> Workload:
    seed = 12345 + 3
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = dy = 16
    a = rng.uniform(0.0, 0.95, size=dx)
    th = np.concatenate([a, np.full(dx, np.log(0.5)), np.full(dy, np.log(1.0))])
    y = simulate_lg(rng, a, np.full(dx, 0.5), np.full(dy, 1.0), None, T)
    # prior N(m0, diag(s0^2)) centred on stable dynamics: under N(0, I) nearly every one of
    # the 16 transition coefficients would put some |a_k| >= 1 (explosive) in each sample
    m0 = np.concatenate([np.full(dx, 0.5), np.full(dx, np.log(0.5)), np.zeros(dy)])
    s0 = np.concatenate([np.full(dx, 0.15), np.full(dx, 0.3), np.full(dy, 0.3)])
    # the paper's step sizes were tuned for its 3-parameter model; with 48 parameters a
    # Langevin step of 0.134 throws samples into explosive dynamics within a few iterations,
    # 0.03 (random walk 0.06) keeps the population alive (scaled with sqrt(200/T))
    gam = {"langevin": 0.03, "rw": 0.06, "hmc": 0.03, "nuts": 0.03}[proposal] * np.sqrt(200.0 / T)
    return Workload("lg16", LG_DIAG, dx, dy, 3 * dx, T, N, M, K, th, y, None, proposal,
                    gam, 780, seed, prior_mean=m0, prior_std=s0)


def lgssm(T=500, N=64, M=250, K=15, proposal="langevin") -> Workload:
    """The linear-Gaussian model of Sec. IV-A: x_t ~ N(mu x_{t-1}, phi^2), y_t ~ N(x_t, sigma^2),
    theta = (mu, phi, sigma) with uniform priors U(-1, 1), U(0, 5), U(0, 5), filtered with the
    optimal proposal; theta* = (0.75, 1, 1); step sizes 0.085 (Langevin) and 0.175 (random walk)."""
    seed = 12345 + 5
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.array([0.75, 1.0, 1.0])
    y = simulate_lg(rng, th[:1], th[1:2], th[2:3], None, T)
    lo = np.array([-1.0, 0.0, 0.0])
    hi = np.array([1.0, 5.0, 5.0])
    return Workload("lgssm", LG_OPT, 1, 1, 3, T, N, M, K, th, y, None, proposal,
                    {"langevin": 0.085, "rw": 0.175, "hmc": 0.085, "nuts": 0.085}[proposal], 781, seed,
                    prior_mean=lo, prior_std=hi, prior_kind=UNIFORM_PRIOR)


ALL = {"lg1": lg1, "lg4": lg4, "sv": sv, "lg16": lg16, "lgssm": lgssm}


def thetas_near(w: Workload, n: int, scale: float = 0.05, seed: int = 4242) -> np.ndarray:
    """n parameter vectors theta* + scale * N(0, I) (FP64), e.g. for likelihood-only calls."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return w.theta_star[None, :] + scale * rng.standard_normal((n, w.D))


def serving_stream(n_jobs=256, rate_hz=50.0, seed=12345 + 4, max_T=1000):
    """Poisson-arrival job list for the serving workload: families of lg1/lg4/sv/lg16,
    T ~ U[50, max_T], N in {256, 1024, 4096}, M in {128, 512, 2048}, own seed and theta*."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    names = ["lg1", "lg4", "sv", "lg16"]
    for j in range(n_jobs):
        t += rng.exponential(1.0 / rate_hz)
        fam = names[int(rng.integers(len(names)))]
        T = int(rng.integers(50, max_T + 1))
        N = int(rng.choice([256, 1024, 4096]))
        M = int(rng.choice([128, 512, 2048]))
        base = ALL[fam]()
        jseed = 100000 + j
        jr = np.random.Generator(np.random.PCG64(jseed))
        th = base.theta_star.copy()
        if base.family == LG_DIAG:
            th[:base.dx] = jr.uniform(0.0, 0.95, size=base.dx)
            y = simulate_lg(jr, th[:base.dx], np.exp(th[base.dx:2 * base.dx]),
                            np.exp(th[2 * base.dx:]), base.H, T)
        else:
            y = simulate_sv(jr, th[0], np.tanh(th[1]), np.exp(th[2]), T)
        wl = replace(base, T=T, N=N, M=M, theta_star=th, y=y, seed=jseed,
                     gamma=step_sizes(T)["langevin"], K=base.K)
        jobs.append((t, wl))
    return jobs
