"""Thin ctypes binding of ``libtauleap.so`` (C ABI in ``include/tauleap.h``).

Argument marshalling only: every step of the simulation runs inside the
CUDA library.  Device arrays are passed as torch CUDA tensors (their
``data_ptr()``), host arrays as numpy arrays.  The library must have been
built (``paper_1309_7695_b300.build``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtauleap.so")

SSA_OK = 0
SSA_EINVAL = -1
SSA_ENOMEM = -2
SSA_EBUSY = -3
SSA_ECUDA = -4
SSA_EUNSUPPORTED = -5

SSA_STATUS_OK = 0
SSA_STATUS_STEP_LIMIT = 1
SSA_STATUS_OVERFLOW = 2
SSA_STATUS_REJECT_LIMIT = 3
SSA_STATUS_INVALID = 4

SSA_JOB_QUEUED = 0
SSA_JOB_RUNNING = 1
SSA_JOB_DONE = 2
SSA_JOB_FAILED = 3

SSA_MODE_TAU_LEAP = 0
SSA_MODE_EXACT = 1
SSA_MODE_CLE = 2
SSA_FP64_REF = 0
SSA_FAST = 1
SSA_LAYOUT_AUTO = 0
SSA_LAYOUT_WARP = 1
SSA_LAYOUT_LANE = 2

# indices of ssa_options.work_counters
SSA_WORK_SELECTIONS = 0
SSA_WORK_TAU_TERMS = 1
SSA_WORK_TAU_SPECIES = 2
SSA_WORK_TAU2 = 3
SSA_WORK_MEANS = 4
SSA_WORK_INV_DRAWS = 5
SSA_WORK_INV_TERMS = 6
SSA_WORK_PTRS_DRAWS = 7
SSA_WORK_PTRS_ITERS = 8
SSA_WORK_PTRS_TESTS = 9
SSA_WORK_COUNTERS = 10
WORK_NAMES = ("selections", "tau_terms", "tau_species", "tau2", "means", "inv_draws", "inv_terms", "ptrs_draws",
              "ptrs_iters", "ptrs_tests")

EXPORTED = [
    "ssa_default_options", "ssa_load_model", "ssa_free_model", "ssa_model_info",
    "ssa_simulate_dev", "ssa_simulate_moments_dev", "ssa_simulate_histograms_dev", "ssa_integrate_rre_dev", "ssa_simulate_dev_noalloc", "ssa_simulate_multi_dev", "ssa_submit_batch", "ssa_poll", "ssa_wait", "ssa_fetch",
    "ssa_release_job", "ssa_last_error", "ssa_abi_version",
    "ssa_server_default_config", "ssa_server_create", "ssa_server_submit", "ssa_server_poll", "ssa_server_wait",
    "ssa_server_fetch", "ssa_server_stats", "ssa_server_destroy", "ssa_server_last_error",
    "ssa_measure_issue_rates",
]


class SsaError(RuntimeError):
    """A call of the C ABI returned a negative SSA_E* code; ``code`` holds it
    and the message is the library's ssa_last_error() text."""

    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class ModelDesc(ctypes.Structure):
    """ssa_model_desc: species and reaction counts and the reactant and
    product CSR arrays (int32)."""

    _fields_ = [
        ("n_species", ctypes.c_int32), ("n_reactions", ctypes.c_int32),
        ("react_ptr", ctypes.c_void_p), ("react_species", ctypes.c_void_p), ("react_coef", ctypes.c_void_p),
        ("prod_ptr", ctypes.c_void_p), ("prod_species", ctypes.c_void_p), ("prod_coef", ctypes.c_void_p),
    ]


class Group(ctypes.Structure):
    """ssa_group: one (network, batch) entry of a persistent multi-network
    launch; every pointer is a device pointer."""

    _fields_ = [
        ("model", ctypes.c_void_p), ("n_sims", ctypes.c_int64), ("sim_offset", ctypes.c_int64),
        ("params", ctypes.c_void_p), ("x0", ctypes.c_void_p), ("t_end", ctypes.c_double),
        ("sample_times", ctypes.c_void_p), ("n_samples", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("samples", ctypes.c_void_p), ("stats", ctypes.c_void_p),
    ]


class Options(ctypes.Structure):
    """ssa_options: method, precision, CGP constants (eps, n_c, the SSA
    fallback factor and block), retry and attempt caps, and launch shape."""

    _fields_ = [
        ("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("eps", ctypes.c_double),
        ("n_c", ctypes.c_int32), ("ssa_block", ctypes.c_int32), ("ssa_factor", ctypes.c_double),
        ("max_halvings", ctypes.c_int32), ("layout", ctypes.c_int32), ("max_attempts", ctypes.c_int64),
        ("block_warps", ctypes.c_int32), ("sims_per_warp", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
        ("reg_cap", ctypes.c_int32), ("work_counters", ctypes.c_void_p),
    ]


class ServerConfig(ctypes.Structure):
    """ssa_server_config: HBM budget, stream slots, requests per launch and
    the options applied to every request."""

    _fields_ = [("max_device_bytes", ctypes.c_int64), ("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("opts", Options)]


class RequestInfo(ctypes.Structure):
    """ssa_request_info: a request's state, the size of the launch it ran in,
    and its submit / admit / done times (seconds since server creation)."""

    _fields_ = [("state", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


STATS_DTYPE = np.dtype([
    ("status", np.int32), ("reserved", np.int32), ("leaps", np.int64), ("rejected", np.int64),
    ("ssa_steps", np.int64), ("firings", np.int64), ("attempts", np.int64), ("t_final", np.float64),
])
assert STATS_DTYPE.itemsize == 56

_lib = None


def lib():
    """Load libtauleap.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1309_7695_b300.build` "
                          "(or __graft_entry__.build()) first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    L.ssa_default_options.argtypes = [ctypes.POINTER(Options)]
    L.ssa_default_options.restype = None
    L.ssa_load_model.argtypes = [ctypes.POINTER(ModelDesc), ctypes.POINTER(vp)]
    L.ssa_free_model.argtypes = [vp]
    L.ssa_model_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.ssa_simulate_dev.argtypes = [vp, i64, i64, vp, vp, f64, vp, i32, u64, ctypes.POINTER(Options), vp, vp, vp]
    L.ssa_simulate_dev_noalloc.argtypes = L.ssa_simulate_dev.argtypes
    L.ssa_integrate_rre_dev.argtypes = [vp, i64, vp, vp, vp, i32, f64, f64, i64, vp, vp, vp]
    L.ssa_simulate_histograms_dev.argtypes = [vp, i64, i64, vp, vp, f64, vp, i32, u64, ctypes.POINTER(Options), i32,
                                              i32, i32, vp, vp, vp]
    L.ssa_simulate_moments_dev.argtypes = [vp, i64, i64, vp, vp, f64, vp, i32, u64, ctypes.POINTER(Options), vp, vp,
                                           vp, vp]
    L.ssa_simulate_multi_dev.argtypes = [i32, ctypes.POINTER(Group), ctypes.POINTER(Options), vp]
    L.ssa_submit_batch.argtypes = [vp, i64, vp, vp, f64, vp, i32, u64, ctypes.POINTER(Options), vp,
                                   ctypes.POINTER(vp)]
    L.ssa_poll.argtypes = [vp, ctypes.POINTER(i32)]
    L.ssa_wait.argtypes = [vp]
    L.ssa_fetch.argtypes = [vp, vp, vp]
    L.ssa_release_job.argtypes = [vp]
    L.ssa_last_error.argtypes = []
    L.ssa_last_error.restype = ctypes.c_char_p
    L.ssa_abi_version.argtypes = []
    L.ssa_server_default_config.argtypes = [ctypes.POINTER(ServerConfig)]
    L.ssa_server_default_config.restype = None
    L.ssa_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.ssa_server_submit.argtypes = [vp, vp, i64, vp, vp, f64, vp, i32, u64, ctypes.POINTER(i64)]
    L.ssa_server_poll.argtypes = [vp, i64, ctypes.POINTER(RequestInfo)]
    L.ssa_server_wait.argtypes = [vp, i64, ctypes.POINTER(RequestInfo)]
    L.ssa_server_fetch.argtypes = [vp, i64, vp, vp]
    L.ssa_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.ssa_server_destroy.argtypes = [vp]
    L.ssa_server_last_error.argtypes = []
    L.ssa_server_last_error.restype = ctypes.c_char_p
    L.ssa_measure_issue_rates.argtypes = [vp, ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(f64)]
    for name in EXPORTED:
        if name not in ("ssa_default_options", "ssa_last_error", "ssa_server_default_config",
                        "ssa_server_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != SSA_OK:
        raise SsaError(rc, lib().ssa_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def ssa_default_options(**overrides) -> Options:
    """The library's default options (tau-leaping, FP64 reference, eps 0.03,
    n_c 10, SSA fallback 10/a0 with blocks of 100), with ``overrides`` set by
    field name."""
    o = Options()
    lib().ssa_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Model:
    """A network loaded on the current CUDA device (ssa_load_model)."""

    def __init__(self, network):
        csr = network.csr()
        self._keep = csr
        d = ModelDesc(network.n_species, network.n_reactions,
                      _ptr(csr["react_ptr"]), _ptr(csr["react_species"]), _ptr(csr["react_coef"]),
                      _ptr(csr["prod_ptr"]), _ptr(csr["prod_species"]), _ptr(csr["prod_coef"]))
        h = ctypes.c_void_p()
        _check(lib().ssa_load_model(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n_species = network.n_species
        self.n_reactions = network.n_reactions

    def close(self):
        """Free the model's device memory (ssa_free_model); idempotent."""
        if self.handle:
            lib().ssa_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ssa_measure_issue_rates(stream=None) -> dict:
    """The device's measured FP64 and FP32 add rates (adds/s over a full-device
    grid) and the latency of one dependent FP64 add in SM cycles."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().ssa_measure_issue_rates(ctypes.c_void_p(handle), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc != SSA_OK:
        raise SsaError(rc, "issue-rate microbenchmark failed")
    return {"fp64_adds_per_s": a.value, "fp32_adds_per_s": b.value, "fp64_add_latency_cycles": c.value}


def ssa_load_model(network) -> Model:
    """Validate ``network`` (an ``inputs.Network``) and upload it to the
    current device."""
    return Model(network)


def ssa_simulate_dev(model: Model, params, x0, t_end, sample_times, samples, stats=None, seed=0,
                     opts=None, sim_offset=0, stream=None):
    """Enqueue simulations on device tensors (torch CUDA tensors).

    params [n, M] float64, x0 [n, N] int32, sample_times [S] float64,
    samples [n, S, N] int32 (output), stats [n * 56] uint8 or None (output).
    ``stream``: a torch.cuda.Stream or raw handle (default: torch's current).
    """
    n = int(params.shape[0]) if params.dim() == 2 else 0
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    o = opts if opts is not None else ssa_default_options()
    _check(lib().ssa_simulate_dev(model.handle, n, int(sim_offset), _ptr(params), _ptr(x0), float(t_end),
                                  _ptr(sample_times), int(sample_times.numel()), int(seed), ctypes.byref(o),
                                  _ptr(samples), _ptr(stats), ctypes.c_void_p(int(handle))))


def ssa_simulate_histograms_dev(model: Model, params, x0, t_end, sample_times, counts, bin_lo, bin_width, n_bins,
                                stats=None, seed=0, opts=None, sim_offset=0, stream=None):
    """Simulate like ssa_simulate_dev but only add every recorded count to its
    (sample time, species) histogram: counts [S, N, n_bins + 2] int64 torch
    CUDA tensor, added to (bin 0 underflow, bins 1..n_bins of width
    bin_width from bin_lo, bin n_bins + 1 overflow)."""
    n = int(params.shape[0]) if params.dim() == 2 else 0
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    o = opts if opts is not None else ssa_default_options()
    _check(lib().ssa_simulate_histograms_dev(model.handle, n, int(sim_offset), _ptr(params), _ptr(x0), float(t_end),
                                             _ptr(sample_times), int(sample_times.numel()), int(seed),
                                             ctypes.byref(o), int(bin_lo), int(bin_width), int(n_bins), _ptr(counts),
                                             _ptr(stats), ctypes.c_void_p(int(handle))))


def ssa_simulate_moments_dev(model: Model, params, x0, t_end, sample_times, mean, var, stats=None, seed=0,
                             opts=None, sim_offset=0, stream=None):
    """Simulate like ssa_simulate_dev but write only the sweep moments:
    mean, var [S, N] float64 torch CUDA tensors (outputs)."""
    n = int(params.shape[0]) if params.dim() == 2 else 0
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    o = opts if opts is not None else ssa_default_options()
    _check(lib().ssa_simulate_moments_dev(model.handle, n, int(sim_offset), _ptr(params), _ptr(x0), float(t_end),
                                          _ptr(sample_times), int(sample_times.numel()), int(seed), ctypes.byref(o),
                                          _ptr(mean), _ptr(var), _ptr(stats), ctypes.c_void_p(int(handle))))


def ssa_integrate_rre_dev(model: Model, params, x0, sample_times, out, stats=None, rtol=1e-8, atol=1e-8,
                          max_steps=1_000_000, stream=None):
    """Reaction-rate-equation trajectories of a batch on device tensors:
    params [n, M] float64, x0 [n, N] int32, sample_times [S] float64,
    out [n, S, N] float64 (output), stats [n * 56] uint8 or None."""
    n = int(params.shape[0]) if params.dim() == 2 else 0
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().ssa_integrate_rre_dev(model.handle, n, _ptr(params), _ptr(x0), _ptr(sample_times),
                                       int(sample_times.numel()), float(rtol), float(atol), int(max_steps),
                                       _ptr(out), _ptr(stats), ctypes.c_void_p(int(handle))))


def ssa_simulate_dev_noalloc(model: Model, params, x0, t_end, sample_times, samples, stats=None, seed=0,
                             opts=None, sim_offset=0, stream=None):
    """Like ssa_simulate_dev, but the library allocates nothing: its work
    counter lives in a static device array shared by all calls (calls that
    overlap on the GPU race on it)."""
    n = int(params.shape[0]) if params.dim() == 2 else 0
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    o = opts if opts is not None else ssa_default_options()
    _check(lib().ssa_simulate_dev_noalloc(model.handle, n, int(sim_offset), _ptr(params), _ptr(x0), float(t_end),
                                          _ptr(sample_times), int(sample_times.numel()), int(seed),
                                          ctypes.byref(o), _ptr(samples), _ptr(stats),
                                          ctypes.c_void_p(int(handle))))


def ssa_simulate_multi_dev(groups, opts=None, stream=None):
    """One persistent launch over several (model, batch) groups.

    ``groups``: sequence of dicts with keys model (Model), params, x0,
    sample_times, samples, stats (torch CUDA tensors; stats may be None),
    t_end, seed and optionally sim_offset, in schedule order."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    arr = (Group * len(groups))()
    for k, g in enumerate(groups):
        p = g["params"]
        arr[k] = Group(g["model"].handle, int(p.shape[0]) if p.dim() == 2 else 0, int(g.get("sim_offset", 0)),
                       _ptr(p), _ptr(g["x0"]), float(g["t_end"]), _ptr(g["sample_times"]),
                       int(g["sample_times"].numel()), 0, int(g["seed"]), _ptr(g["samples"]),
                       _ptr(g.get("stats")))
    o = opts if opts is not None else ssa_default_options()
    _check(lib().ssa_simulate_multi_dev(len(groups), arr, ctypes.byref(o), ctypes.c_void_p(int(handle))))


class Job:
    """A host-buffer job (ssa_submit_batch / ssa_poll / ssa_fetch / ssa_release_job)."""

    def __init__(self, model: Model, handle, n_sims, n_samples):
        self.model, self.handle, self.n_sims, self.n_samples = model, handle, n_sims, n_samples

    def poll(self) -> int:
        """SSA_JOB_RUNNING, SSA_JOB_DONE or SSA_JOB_FAILED, without blocking."""
        st = ctypes.c_int32()
        _check(lib().ssa_poll(self.handle, ctypes.byref(st)))
        return st.value

    def wait(self):
        """Block until the job's work is complete."""
        _check(lib().ssa_wait(self.handle))

    def fetch(self, samples=None, stats=None):
        """Wait, then copy samples [n][S][N] int32 and stats [n] to host arrays
        (allocated when not given); returns (samples, stats)."""
        if samples is None:
            samples = np.empty((self.n_sims, self.n_samples, self.model.n_species), dtype=np.int32)
        if stats is None:
            stats = np.empty(self.n_sims, dtype=STATS_DTYPE)
        _check(lib().ssa_fetch(self.handle, _ptr(samples), _ptr(stats)))
        return samples, stats

    def release(self):
        """Wait for the job and free everything it owns; idempotent."""
        if self.handle:
            _check(lib().ssa_release_job(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def ssa_submit_batch(model: Model, params, x0, t_end, sample_times, seed=0, opts=None, stream=None) -> Job:
    """Host-buffer job: params [n, M] float64, x0 [n, N] int32 and sample
    times [S] are copied to device memory the job owns, and the simulation is
    enqueued on ``stream`` (default: a stream of the job's own)."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    T = np.ascontiguousarray(sample_times, dtype=np.float64)
    n = int(params.shape[0])
    o = opts if opts is not None else ssa_default_options()
    h = ctypes.c_void_p()
    s = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    _check(lib().ssa_submit_batch(model.handle, n, _ptr(params), _ptr(x0), float(t_end), _ptr(T), int(T.size),
                                  int(seed), ctypes.byref(o), s, ctypes.byref(h)))
    return Job(model, h, n, int(T.size))


def simulate_host(network, params, x0, t_end, sample_times, seed=0, opts=None):
    """Convenience: load, submit, fetch and release; returns (samples, stats)."""
    m = Model(network)
    try:
        j = ssa_submit_batch(m, params, x0, t_end, sample_times, seed, opts)
        try:
            return j.fetch()
        finally:
            j.release()
    finally:
        m.close()


def _scheck(rc):
    if rc != SSA_OK:
        raise SsaError(rc, lib().ssa_server_last_error().decode())


class Server:
    """Continuous-batching request server (ssa_server_*)."""

    def __init__(self, max_device_bytes=0, n_streams=4, max_batch=16, opts=None):
        c = ServerConfig()
        lib().ssa_server_default_config(ctypes.byref(c))
        c.max_device_bytes = int(max_device_bytes)
        c.n_streams = int(n_streams)
        c.max_batch = int(max_batch)
        if opts is not None:
            c.opts = opts
        h = ctypes.c_void_p()
        _scheck(lib().ssa_server_create(ctypes.byref(c), ctypes.byref(h)))
        self.handle = h
        self._shapes = {}

    def submit(self, model, params, x0, t_end, sample_times, seed=0) -> int:
        """Queue a request with host inputs (copied before returning); returns
        its ticket.  Simulation r uses the stream (seed, r)."""
        params = np.ascontiguousarray(params, dtype=np.float64)
        x0 = np.ascontiguousarray(x0, dtype=np.int32)
        T = np.ascontiguousarray(sample_times, dtype=np.float64)
        t = ctypes.c_int64()
        _scheck(lib().ssa_server_submit(self.handle, model.handle, int(params.shape[0]), _ptr(params), _ptr(x0),
                                        float(t_end), _ptr(T), int(T.size), int(seed), ctypes.byref(t)))
        self._shapes[t.value] = (int(params.shape[0]), int(T.size), model.n_species)
        return t.value

    def poll(self, ticket) -> RequestInfo:
        """The request's state and times, without blocking."""
        info = RequestInfo()
        _scheck(lib().ssa_server_poll(self.handle, int(ticket), ctypes.byref(info)))
        return info

    def wait(self, ticket) -> RequestInfo:
        """Block until the request's launch has completed."""
        info = RequestInfo()
        _scheck(lib().ssa_server_wait(self.handle, int(ticket), ctypes.byref(info)))
        return info

    def fetch(self, ticket):
        """Wait for the request, copy out (samples [n][S][N], stats [n]), free
        its device memory and forget the ticket."""
        n, S, N = self._shapes[ticket]
        samples = np.empty((n, S, N), dtype=np.int32)
        stats = np.empty(n, dtype=STATS_DTYPE)
        _scheck(lib().ssa_server_fetch(self.handle, int(ticket), _ptr(samples), _ptr(stats)))
        del self._shapes[ticket]
        return samples, stats

    def stats(self):
        """Launches issued, requests waiting for admission, admitted bytes."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _scheck(lib().ssa_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"launches": a.value, "queued": b.value, "device_bytes_in_use": c.value}

    def close(self):
        """Finish queued and running requests and free everything; idempotent."""
        if self.handle:
            lib().ssa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
