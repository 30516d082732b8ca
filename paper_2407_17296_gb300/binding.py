"""Thin ctypes binding of the C ABI in ``include/smc2.h`` (argument marshalling only).

Every computation runs in the CUDA library ``libsmc2.so``; this module only
converts Python/torch arguments into plain pointers and sizes.  torch supplies
device memory and streams.  If the library was not built, ``load()`` raises:
there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmc2.so")

SMC2_OK = 0
SMC2_PENDING = 1
ERRORS = {-1: "SMC2_E_INVAL", -2: "SMC2_E_NOMEM", -3: "SMC2_E_CUDA", -4: "SMC2_E_TIMEOUT",
          -5: "SMC2_E_NOTFOUND", -6: "SMC2_E_BUSY"}
LG_DIAG, SV, LG_OPT = 0, 1, 2
PRIOR_GAUSSIAN, PRIOR_UNIFORM = 0, 1
RW, LANGEVIN, HMC, NUTS = 0, 1, 2, 3
PROPOSALS = {"rw": RW, "langevin": LANGEVIN, "hmc": HMC, "nuts": NUTS}
NUTS_REVERSAL, NUTS_MOMENTUM_REVERSAL = 0, 1
SYSTEMATIC, MULTINOMIAL = 0, 1

# every symbol include/smc2.h declares
EXPORTS = ("smc2_config_init", "smc2_create", "pf_loglik_grad", "pf_loglik_grad_rows",
           "pf_loglik_grad_host", "smc2_step", "smc2_step_filters", "smc2_step_update", "smc2_run", "smc2_set_step_timing", "smc2_get_step_timing", "smc2_get_samples", "smc2_get_state",
           "smc2_get_trace", "smc2_set_observations", "smc2_footprint", "smc2_destroy",
           "smc2_autotune", "smc2_get_launch", "smc2_set_launch", "smc2_get_status", "smc2_selftest_bounded_wait", "smc2_kernel_launches", "smc2_last_error", "smc2_server_create",
           "smc2_submit", "smc2_poll", "smc2_cancel", "smc2_server_destroy",
           "pf_loglik_grad_static", "pf_static_get_status", "smc2_get_stream", "smc2_selftest_crn",
           "smc2_batch_create", "smc2_batch_step", "smc2_batch_destroy", "smc2_server_set_fused",
           "smc2_get_nuts_trace", "smc2_set_point_trace", "smc2_get_point_trace")


class Config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("model_family", ctypes.c_int32),
        ("d_x", ctypes.c_int32),
        ("d_y", ctypes.c_int32),
        ("H", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("y_on_device", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("D", ctypes.c_int32),
        ("prior_mean", ctypes.c_void_p),
        ("prior_std", ctypes.c_void_p),
        ("proposal", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("K_iters", ctypes.c_int32),
        ("pf_resample", ctypes.c_int32),
        ("ess_frac", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("ckpt_every", ctypes.c_int32),
        ("particles_per_thread", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("prior_kind", ctypes.c_int32),
        ("hmc_steps", ctypes.c_int32),
        ("nuts_max_depth", ctypes.c_int32),
        ("nuts_weight", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32),
        ("resampled", ctypes.c_int32),
        ("ess", ctypes.c_double),
        ("l_k", ctypes.c_double),
        ("max_logw", ctypes.c_double),
        ("mean", ctypes.c_void_p),
        ("recycled_mean", ctypes.c_void_p),
        ("pf_near_ties", ctypes.c_int64),
        ("pf_resample_steps", ctypes.c_int64),
        ("outer_near_ties", ctypes.c_int64),
    ]


def _stats_dict(st, mean, rec):
    return {"k": st.k, "resampled": bool(st.resampled), "ess": st.ess, "l_k": st.l_k,
            "max_logw": st.max_logw, "mean": mean, "recycled_mean": rec,
            "pf_near_ties": int(st.pf_near_ties), "pf_resample_steps": int(st.pf_resample_steps),
            "outer_near_ties": int(st.outer_near_ties)}


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("latency_s", ctypes.c_double),
        ("queue_s", ctypes.c_double),
        ("theta", ctypes.c_void_p),
        ("logw", ctypes.c_void_p),
        ("recycled_mean", ctypes.c_void_p),
    ]


class Smc2Error(RuntimeError):
    pass


_lib = None


def load(path: str = LIB_PATH):
    """Load libsmc2.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise Smc2Error(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, u32, u64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    sig = {
        "smc2_config_init": (None, [ctypes.POINTER(Config)]),
        "smc2_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(vp)]),
        "pf_loglik_grad": (ctypes.c_int, [vp, dp, ctypes.c_int, u32, dp, dp]),
        "pf_loglik_grad_rows": (ctypes.c_int, [vp, dp, ctypes.c_int, u32, u32, dp, dp]),
        "pf_loglik_grad_host": (ctypes.c_int, [vp, dp, ctypes.c_int, u32, dp, dp]),
        "smc2_step": (ctypes.c_int, [vp, ctypes.POINTER(Stats)]),
        "smc2_step_filters": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, dp]),
        "smc2_run": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(Stats)]),
        "smc2_set_step_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "smc2_get_step_timing": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "smc2_step_update": (ctypes.c_int, [vp, dp, dp, ctypes.POINTER(Stats)]),
        "smc2_get_samples": (ctypes.c_int, [vp, dp, dp]),
        "smc2_get_state": (ctypes.c_int, [vp, dp, dp]),
        "smc2_get_trace": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "smc2_get_nuts_trace": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "smc2_set_point_trace": (ctypes.c_int, [vp, ctypes.c_int]),
        "smc2_get_point_trace": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "smc2_set_observations": (ctypes.c_int, [vp, vp]),
        "smc2_footprint": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]),
        "smc2_destroy": (ctypes.c_int, [vp]),
        "smc2_autotune": (ctypes.c_int, [ctypes.POINTER(Config), dp, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
        "smc2_get_launch": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
        "smc2_set_launch": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_int)]),
        "smc2_get_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
        "smc2_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "smc2_kernel_launches": (u64, []),
        "smc2_last_error": (ctypes.c_char_p, []),
        "smc2_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]),
        "smc2_submit": (ctypes.c_int, [vp, ctypes.POINTER(Config), ctypes.POINTER(u64)]),
        "smc2_poll": (ctypes.c_int, [vp, u64, ctypes.POINTER(Result)]),
        "smc2_cancel": (ctypes.c_int, [vp, u64]),
        "smc2_server_destroy": (ctypes.c_int, [vp]),
        "pf_loglik_grad_static": (ctypes.c_int, [ctypes.POINTER(Config), dp, ctypes.c_int, u32, u32,
                                                 dp, dp]),
        "pf_static_get_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
        "smc2_get_stream": (ctypes.c_int, [vp, ctypes.POINTER(vp)]),
        "smc2_selftest_crn": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp, vp, vp]),
        "smc2_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp)]),
        "smc2_batch_step": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(Stats)]),
        "smc2_batch_destroy": (ctypes.c_int, [vp]),
        "smc2_server_set_fused": (ctypes.c_int, [vp, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    c = Config()
    lib.smc2_config_init(ctypes.byref(c))
    if c.struct_size != ctypes.sizeof(Config):
        raise Smc2Error(f"smc2_config layout mismatch: C {c.struct_size} vs ctypes {ctypes.sizeof(Config)}")
    _lib = lib
    return lib


def check(rc: int, what: str = "") -> int:
    if rc < 0:
        msg = load().smc2_last_error().decode(errors="replace")
        raise Smc2Error(f"{what}: {ERRORS.get(rc, rc)}: {msg}")
    return rc


def last_error() -> str:
    return load().smc2_last_error().decode(errors="replace")


def kernel_launches() -> int:
    return int(load().smc2_kernel_launches())


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def make_config(family, dx, dy, T, N, M, D, y, H=None, prior_mean=None, prior_std=None,
                proposal=LANGEVIN, gamma=0.1, K_iters=10, pf_resample=SYSTEMATIC, ess_frac=0.5,
                seed=777, ckpt_every=0, particles_per_thread=0, stream=None, y_on_device=False,
                prior_kind=PRIOR_GAUSSIAN, hmc_steps=1, nuts_max_depth=3, nuts_weight=NUTS_REVERSAL):
    """Build a Config; numpy arrays referenced by it are kept alive on the returned object."""
    import numpy as np
    lib = load()
    c = Config()
    lib.smc2_config_init(ctypes.byref(c))
    keep = []
    c.model_family, c.d_x, c.d_y = int(family), int(dx), int(dy)
    c.T, c.N, c.M, c.D = int(T), int(N), int(M), int(D)
    if y_on_device:
        c.y = ctypes.c_void_p(y.data_ptr()).value
        c.y_on_device = 1
        keep.append(y)
    else:
        ya = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
        keep.append(ya)
        c.y = ya.ctypes.data
    if H is not None:
        Ha = np.ascontiguousarray(np.asarray(H, dtype=np.float32))
        keep.append(Ha)
        c.H = Ha.ctypes.data
    for name, arr in (("prior_mean", prior_mean), ("prior_std", prior_std)):
        if arr is not None:
            a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
            keep.append(a)
            setattr(c, name, a.ctypes.data)
    c.proposal = int(proposal)
    c.gamma = float(gamma)
    c.K_iters = int(K_iters)
    c.pf_resample = int(pf_resample)
    c.ess_frac = float(ess_frac)
    c.seed = int(seed)
    c.ckpt_every = int(ckpt_every)
    c.particles_per_thread = int(particles_per_thread)
    c.stream = stream
    c.prior_kind = int(prior_kind)
    c.hmc_steps = int(hmc_steps)
    c.nuts_max_depth = int(nuts_max_depth)
    c.nuts_weight = int(nuts_weight)
    c._keep = keep
    return c


class Handle:
    """One device-resident SMC^2 job (smc2_create ... smc2_destroy)."""

    def __init__(self, cfg: Config):
        self.lib = load()
        self.cfg = cfg
        self.D, self.N, self.T, self.M = cfg.D, cfg.N, cfg.T, cfg.M
        h = ctypes.c_void_p()
        check(self.lib.smc2_create(ctypes.byref(cfg), ctypes.byref(h)), "smc2_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            check(self.lib.smc2_destroy(self.h), "smc2_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- hot path ------------------------------------------------------------
    def pf_loglik_grad(self, theta, iteration, loglik, grad=None, row0=0):
        """theta: (n, D) float64 CUDA tensor; loglik: (n,) float64; grad: (n, D) float64 or None."""
        n = int(theta.shape[0])
        check(self.lib.pf_loglik_grad_rows(self.h, _ptr(theta), n, int(iteration), int(row0),
                                           _ptr(loglik), _ptr(grad)), "pf_loglik_grad")

    def pf_loglik_grad_host(self, theta, iteration, loglik, grad=None):
        """numpy float64 host arrays in and out (copies inside the call)."""
        n = int(theta.shape[0])
        check(self.lib.pf_loglik_grad_host(self.h, _ptr(theta), n, int(iteration), _ptr(loglik),
                                           _ptr(grad)), "pf_loglik_grad_host")

    def step(self, want_means=True):
        import numpy as np
        st = Stats()
        mean = np.zeros(self.D)
        rec = np.zeros(self.D)
        if want_means:
            st.mean = mean.ctypes.data
            st.recycled_mean = rec.ctypes.data
        check(self.lib.smc2_step(self.h, ctypes.byref(st)), "smc2_step")
        return _stats_dict(st, mean, rec)

    def run(self, K, want_means=True):
        """K iterations back to back; statistics of the last one."""
        import numpy as np
        st = Stats()
        mean = np.zeros(self.D)
        rec = np.zeros(self.D)
        if want_means:
            st.mean = mean.ctypes.data
            st.recycled_mean = rec.ctypes.data
        check(self.lib.smc2_run(self.h, int(K), ctypes.byref(st)), "smc2_run")
        return _stats_dict(st, mean, rec)

    def set_step_timing(self, on=True):
        check(self.lib.smc2_set_step_timing(self.h, 1 if on else 0), "smc2_set_step_timing")

    def step_timing(self):
        """Mean (forward ms, adjoint ms) of the filter passes of the iterations run since the
        last query (device events); (both passes, -1) when the handle overlaps the passes of
        two halves of its filters."""
        ms = (ctypes.c_float * 2)()
        check(self.lib.smc2_get_step_timing(self.h, ms), "smc2_get_step_timing")
        return float(ms[0]), float(ms[1])

    def step_filters(self, row0, n, loglik, grad):
        """Propose for all N samples and run the filters of rows row0 .. row0+n-1 into the
        device tensors loglik [n] and grad [n][D] (FP64); asynchronous."""
        check(self.lib.smc2_step_filters(self.h, int(row0), int(n), _ptr(loglik), _ptr(grad)),
              "smc2_step_filters")

    def step_update(self, loglik_all, grad_all, want_means=True):
        """Complete the iteration from the filter outputs of all N rows (device tensors)."""
        import numpy as np
        st = Stats()
        mean = np.zeros(self.D)
        rec = np.zeros(self.D)
        if want_means:
            st.mean = mean.ctypes.data
            st.recycled_mean = rec.ctypes.data
        check(self.lib.smc2_step_update(self.h, _ptr(loglik_all), _ptr(grad_all), ctypes.byref(st)),
              "smc2_step_update")
        return _stats_dict(st, mean, rec)

    def samples(self):
        import numpy as np
        th = np.zeros((self.N, self.D))
        lw = np.zeros(self.N)
        check(self.lib.smc2_get_samples(self.h, _ptr(th), _ptr(lw)), "smc2_get_samples")
        return th, lw

    def state(self):
        import numpy as np
        ll = np.zeros(self.N)
        g = np.zeros((self.N, self.D))
        check(self.lib.smc2_get_state(self.h, _ptr(ll), _ptr(g)), "smc2_get_state")
        return ll, g

    def trace(self):
        import numpy as np
        anc = np.zeros((self.N, self.T, self.M), dtype=np.uint16)
        flag = np.zeros((self.N, self.T), dtype=np.uint8)
        oanc = np.zeros(self.N, dtype=np.int32)
        ores = ctypes.c_int32(0)
        check(self.lib.smc2_get_trace(self.h, _ptr(anc), _ptr(flag), _ptr(oanc), ctypes.byref(ores)),
              "smc2_get_trace")
        return anc, flag, oanc, bool(ores.value)

    def set_point_trace(self, on=True):
        check(self.lib.smc2_set_point_trace(self.h, int(bool(on))), "smc2_set_point_trace")

    def point_trace(self, point):
        """(pf_anc [N][T][M], pf_flag [N][T]) of leapfrog point `point` of the last iteration."""
        import numpy as np
        anc = np.zeros((self.N, self.T, self.M), dtype=np.uint16)
        flag = np.zeros((self.N, self.T), dtype=np.uint8)
        check(self.lib.smc2_get_point_trace(self.h, int(point), _ptr(anc), _ptr(flag)), "smc2_get_point_trace")
        return anc, flag

    def nuts_trace(self):
        """Per-sample decisions of the last NUTS move: {"sel": [N] uint64, "merge": [N] uint32,
        "stop_point": [N], "stop_kind": [N]} (smc2_get_nuts_trace)."""
        import numpy as np
        sel = np.zeros(self.N, dtype=np.uint64)
        merge = np.zeros(self.N, dtype=np.uint32)
        sp = np.zeros(self.N, dtype=np.int32)
        sk = np.zeros(self.N, dtype=np.int32)
        check(self.lib.smc2_get_nuts_trace(self.h, _ptr(sel), _ptr(merge), _ptr(sp), _ptr(sk)),
              "smc2_get_nuts_trace")
        return {"sel": sel, "merge": merge, "stop_point": sp, "stop_kind": sk}

    def stream_ptr(self):
        """The cudaStream_t (an int) on which the handle enqueues its work."""
        p = ctypes.c_void_p()
        check(self.lib.smc2_get_stream(self.h, ctypes.byref(p)), "smc2_get_stream")
        return int(p.value or 0)

    def status(self, clear=False):
        """Device status word of the handle's kernels (0 = fine)."""
        st = ctypes.c_int(0)
        check(self.lib.smc2_get_status(self.h, ctypes.byref(st), int(bool(clear))), "smc2_get_status")
        return st.value

    def launch(self):
        """(forward particles/thread, forward register cap, adjoint particles/thread,
        adjoint register cap, checkpoint interval) chosen for this handle."""
        out = (ctypes.c_int * 5)()
        check(self.lib.smc2_get_launch(self.h, out), "smc2_get_launch")
        return tuple(out)

    def set_observations(self, y):
        import numpy as np
        ya = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
        check(self.lib.smc2_set_observations(self.h, _ptr(ya)), "smc2_set_observations")


class Batch:
    """Fused iterations of several handles (smc2_batch_create / smc2_batch_step)."""

    def __init__(self, max_jobs: int):
        self.lib = load()
        b = ctypes.c_void_p()
        check(self.lib.smc2_batch_create(int(max_jobs), ctypes.byref(b)), "smc2_batch_create")
        self.b = b

    def step(self, handles, want_means=True):
        """One SMC^2 iteration of every handle (fused filter passes); list of stats dicts."""
        import numpy as np
        n = len(handles)
        arr = (ctypes.c_void_p * max(n, 1))(*[h.h.value for h in handles])
        st = (Stats * max(n, 1))()
        means = []
        for i, h in enumerate(handles):
            m, r = np.zeros(h.D), np.zeros(h.D)
            if want_means:
                st[i].mean, st[i].recycled_mean = m.ctypes.data, r.ctypes.data
            means.append((m, r))
        check(self.lib.smc2_batch_step(self.b, arr, n, st), "smc2_batch_step")
        return [_stats_dict(st[i], means[i][0], means[i][1]) for i in range(n)]

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            check(self.lib.smc2_batch_destroy(self.b), "smc2_batch_destroy")
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request loop (smc2_server_create ... smc2_server_destroy)."""

    def __init__(self, hbm_budget: int, max_active: int = 8):
        self.lib = load()
        s = ctypes.c_void_p()
        check(self.lib.smc2_server_create(int(hbm_budget), int(max_active), ctypes.byref(s)),
              "smc2_server_create")
        self.s = s
        self.D = {}
        self.N = {}

    def set_fused(self, on=True):
        """Fused batching of ready jobs (default) or one stream a job."""
        check(self.lib.smc2_server_set_fused(self.s, 1 if on else 0), "smc2_server_set_fused")

    def submit(self, cfg: Config) -> int:
        jid = ctypes.c_uint64(0)
        check(self.lib.smc2_submit(self.s, ctypes.byref(cfg), ctypes.byref(jid)), "smc2_submit")
        self.D[jid.value] = cfg.D
        self.N[jid.value] = cfg.N
        return jid.value

    def poll(self, job_id: int):
        """None while pending; else a dict with the job's results (the job is released)."""
        import numpy as np
        D, N = self.D.get(job_id, 1), self.N.get(job_id, 1)
        r = Result()
        th = np.zeros((N, D))
        lw = np.zeros(N)
        rec = np.zeros(D)
        r.theta, r.logw, r.recycled_mean = th.ctypes.data, lw.ctypes.data, rec.ctypes.data
        rc = check(self.lib.smc2_poll(self.s, int(job_id), ctypes.byref(r)), "smc2_poll")
        if rc == SMC2_PENDING:
            return None
        return {"status": r.status, "K": r.K, "latency_s": r.latency_s, "queue_s": r.queue_s,
                "theta": th, "logw": lw, "recycled_mean": rec}

    def cancel(self, job_id: int):
        check(self.lib.smc2_cancel(self.s, int(job_id)), "smc2_cancel")

    def close(self):
        if getattr(self, "s", None) is not None and self.s.value:
            check(self.lib.smc2_server_destroy(self.s), "smc2_server_destroy")
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune(cfg: Config, theta=None):
    """Time the launch variants for cfg's shape on the current device (optionally on the
    given [N][D] parameters) and cache the fastest; returns (particles/thread, ckpt)."""
    import numpy as np
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    ppt, kc = ctypes.c_int(0), ctypes.c_int(0)
    check(load().smc2_autotune(ctypes.byref(cfg), _ptr(th), ctypes.byref(ppt), ctypes.byref(kc)),
          "smc2_autotune")
    return ppt.value, kc.value


def set_launch(cfg: Config, launch):
    """Pin (forward ppt, forward regs, adjoint ppt, adjoint regs, checkpoint interval) for
    cfg's shape; handles created afterwards use it."""
    arr = (ctypes.c_int * 5)(*[int(v) for v in launch])
    check(load().smc2_set_launch(ctypes.byref(cfg), arr), "smc2_set_launch")


def selftest_bounded_wait(polls=1000) -> bool:
    """Run a block whose wait nothing completes; True if the bounded wait reported it."""
    out = ctypes.c_int(0)
    check(load().smc2_selftest_bounded_wait(int(polls), ctypes.byref(out)), "smc2_selftest_bounded_wait")
    return bool(out.value)


def selftest_crn(ctr, key, want=("words", "u", "z")):
    """The filter kernels' Philox4x32-10 words, (0,1] uniforms and Box-Muller normals for the
    counters ctr [n][4] and keys key [n][4] = (seed_lo, seed_hi, iter, row) (uint32 numpy
    arrays, copied to the device); returns numpy arrays [n][4]."""
    import numpy as np
    import torch
    c = torch.as_tensor(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32), device="cuda")
    k = torch.as_tensor(np.ascontiguousarray(key, dtype=np.uint32).view(np.int32), device="cuda")
    n = int(c.shape[0])
    words = torch.zeros((n, 4), dtype=torch.int32, device="cuda") if "words" in want else None
    u = torch.zeros((n, 4), dtype=torch.float32, device="cuda") if "u" in want else None
    z = torch.zeros((n, 4), dtype=torch.float32, device="cuda") if "z" in want else None
    stream = torch.cuda.current_stream().cuda_stream
    check(load().smc2_selftest_crn(_ptr(c), _ptr(k), n, _ptr(words), _ptr(u), _ptr(z),
                                   ctypes.c_void_p(stream)), "smc2_selftest_crn")
    out = {}
    if words is not None:
        out["words"] = words.cpu().numpy().view(np.uint32)
    if u is not None:
        out["u"] = u.cpu().numpy()
    if z is not None:
        out["z"] = z.cpu().numpy()
    return out


def static_status(stream=None, clear=False) -> int:
    """Status word of the last pf_loglik_grad_static call on the current device (0 = fine)."""
    st = ctypes.c_int(0)
    check(load().pf_static_get_status(None if stream is None else ctypes.c_void_p(int(stream)),
                                      ctypes.byref(st), int(bool(clear))), "pf_static_get_status")
    return st.value


def footprint(cfg: Config) -> int:
    b = ctypes.c_size_t(0)
    check(load().smc2_footprint(ctypes.byref(cfg), ctypes.byref(b)), "smc2_footprint")
    return int(b.value)


def config_for(workload, **kw):
    """Config for a workloads.Workload (sizes, data and step size taken from it)."""
    args = dict(proposal=PROPOSALS[workload.proposal], gamma=workload.gamma, K_iters=workload.K,
                seed=workload.seed, prior_mean=workload.prior_mean, prior_std=workload.prior_std,
                prior_kind=getattr(workload, "prior_kind", PRIOR_GAUSSIAN),
                hmc_steps=getattr(workload, "hmc_steps", 1),
                nuts_max_depth=getattr(workload, "nuts_depth", 3),
                nuts_weight=getattr(workload, "nuts_weight", NUTS_REVERSAL))
    args.update(kw)
    return make_config(workload.family, workload.dx, workload.dy, workload.T, workload.N, workload.M,
                       workload.D, workload.y, workload.H, **args)
