"""ctypes binding of libpqmc.so (argument marshalling only).

Every entry point of ``include/pqmc.h`` is reachable under the same name.
Nothing here computes any step of the sweep: the library does, on the GPU.
``load()`` raises when the library has not been built; there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpqmc.so")

OK, EINVAL, ENOMEM, ECUDA, ESTAB, ENAN, ETIMEOUT = range(7)
STATUS = {0: "PQMC_OK", 1: "PQMC_EINVAL", 2: "PQMC_ENOMEM", 3: "PQMC_ECUDA", 4: "PQMC_ESTAB",
          5: "PQMC_ENAN", 6: "PQMC_ETIMEOUT"}
FP64, FP32, BF16X3 = 0, 1, 2
HONEYCOMB, SQUARE, HONEYCOMB_TV = 0, 1, 2


class Lattice(C.Structure):
    _fields_ = [("kind", C.c_int), ("Lx", C.c_int), ("Ly", C.c_int), ("t", C.c_double), ("tp", C.c_double)]


class Trial(C.Structure):
    _fields_ = [("g", C.c_double), ("M_N", C.c_double), ("N_up", C.c_int), ("N_dn", C.c_int),
                ("tiebreak", C.c_double)]


class ChainSpec(C.Structure):
    _fields_ = [("lattice", Lattice), ("U", C.c_double), ("dtau", C.c_double), ("two_theta", C.c_double),
                ("trial", Trial)]


class Opts(C.Structure):
    _fields_ = [("n_stab", C.c_int), ("delay_k", C.c_int), ("prec", C.c_int), ("seed", C.c_uint64),
                ("n_chains", C.c_int), ("chain_offset", C.c_int), ("accept_log", C.c_int),
                ("max_meas", C.c_int), ("stream", C.c_void_p), ("cta_threads", C.c_int), ("dense_chains", C.c_int),
                ("dg_fp64", C.c_int), ("spread", C.c_int)]


# columns of a measurement record: sign of the weight, E/site, docc/site,
# kinetic/site, running sign, S_AFM
RECORD = 6


class Obs(C.Structure):
    _fields_ = [("E", C.c_double), ("E_err", C.c_double), ("docc", C.c_double), ("docc_err", C.c_double),
                ("sign", C.c_double), ("sign_err", C.c_double), ("accept", C.c_double), ("max_dG", C.c_double),
                ("n_meas", C.c_long), ("s_afm", C.c_double), ("s_afm_err", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tune(C.Structure):
    _fields_ = [("delay_k", C.c_int), ("cta_threads", C.c_int), ("ms_per_sweep", C.c_double),
                ("proxy_ltau", C.c_int), ("n_candidates", C.c_int), ("cand_delay_k", C.c_int * 32),
                ("cand_cta_threads", C.c_int * 32), ("cand_ms", C.c_double * 32), ("from_cache", C.c_int)]

    def as_dict(self):
        n = self.n_candidates
        return {"delay_k": self.delay_k, "cta_threads": self.cta_threads, "ms_per_sweep": self.ms_per_sweep,
                "proxy_ltau": self.proxy_ltau, "from_cache": bool(self.from_cache),
                "candidates": [{"delay_k": self.cand_delay_k[i], "cta_threads": self.cand_cta_threads[i],
                                "ms_per_sweep": self.cand_ms[i]} for i in range(n)]}


_lib = None

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("pqmc_init", C.c_int, [C.POINTER(Lattice), C.c_double, C.c_double, C.c_double, C.POINTER(Trial),
                            C.POINTER(Opts), C.POINTER(C.c_void_p)]),
    ("pqmc_init_batch", C.c_int, [C.c_int, C.POINTER(ChainSpec), C.POINTER(Opts), C.POINTER(C.c_void_p)]),
    ("pqmc_sweep", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("pqmc_synchronize", C.c_int, [C.c_void_p]),
    ("pqmc_measure", C.c_int, [C.c_void_p, C.c_int, C.POINTER(Obs)]),
    ("pqmc_get_measurements", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_long)]),
    ("pqmc_get_last_records", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("pqmc_set_fields", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int8)]),
    ("pqmc_get_fields", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int8)]),
    ("pqmc_get_green", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    ("pqmc_get_green_at", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    ("pqmc_checkpoint", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    ("pqmc_restore", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("pqmc_get_weight", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    ("pqmc_write_run_log", C.c_int, [C.c_void_p, C.c_char_p]),
    ("pqmc_get_accept_log", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint8), C.c_long]),
    ("pqmc_get_stab_errors", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_long)]),
    ("pqmc_get_phase_cycles", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_longlong)]),
    ("pqmc_get_dims", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    ("pqmc_num_chains", C.c_int, [C.c_void_p]),
    ("pqmc_launch_count", C.c_long, [C.c_void_p]),
    ("pqmc_device_bytes", C.c_size_t, [C.c_void_p]),
    ("pqmc_upload_bytes", C.c_size_t, [C.c_void_p]),
    ("pqmc_last_error", C.c_char_p, [C.c_void_p]),
    ("pqmc_free", None, [C.c_void_p]),
    ("pqmc_host_model", C.c_int, [C.POINTER(Lattice), C.c_double, C.POINTER(Trial), C.c_int,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    ("pqmc_host_eigh", C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("pqmc_green_noalloc", C.c_int, [C.POINTER(ChainSpec), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    ("pqmc_host_jackknife", C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("pqmc_inject_error", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("pqmc_autotune", C.c_int, [C.c_int, C.POINTER(ChainSpec), C.POINTER(Opts), C.POINTER(Tune)]),
    ("pqmc_get_launch", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("pqmc_probe_pipes", C.c_int, [C.POINTER(C.c_double)]),
    ("pqmc_test_tc_gemm", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
]


def load(path=LIB_PATH):
    """Load libpqmc.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpqmc.so is not built (%s); run paper_2303_13403_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class PQMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _check(st, ctx=None):
    if st != OK:
        msg = load().pqmc_last_error(ctx).decode()
        raise PQMCError(st, msg)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice_of(spec):
    return Lattice(spec.kind, spec.Lx, spec.Ly, spec.t, spec.tp)


def trial_of(spec):
    return Trial(spec.g, spec.M_N, spec.n_up, spec.n_dn, spec.tiebreak)


def chain_spec_of(spec):
    return ChainSpec(lattice_of(spec), spec.U, spec.dtau, spec.two_theta, trial_of(spec))


class Context:
    """One libpqmc context: a batch of chains on the GPU."""

    def __init__(self, specs, prec=FP64, seed=1, n_stab=10, delay_k=32, chain_offset=0, accept_log=0,
                 max_meas=0, stream=None, cta_threads=0, dense_chains=0, dg_fp64=0, spread=0):
        """delay_k = 0 lets the library's autotuner pick the delayed-update
        block (and the CTA shape when cta_threads is 0); spread = 1 sweeps a
        few large chains with grid-wide kernels (pqmc_opts.spread)."""
        lib = load()
        specs = list(specs)
        arr = (ChainSpec * len(specs))(*[chain_spec_of(s) for s in specs])
        opts = Opts(n_stab, delay_k, prec, seed, len(specs), chain_offset, accept_log, max_meas,
                    C.c_void_p(stream) if stream else None, cta_threads, dense_chains, dg_fp64, spread)
        h = C.c_void_p()
        _check(lib.pqmc_init_batch(len(specs), arr, C.byref(opts), C.byref(h)))
        self._h = h
        self.specs = specs
        self.prec = prec
        self.n_chains = len(specs)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().pqmc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1, measure=True):
        _check(load().pqmc_sweep(self._h, n, 1 if measure else 0), self._h)

    def synchronize(self):
        _check(load().pqmc_synchronize(self._h), self._h)

    def measure(self, chain=-1):
        o = Obs()
        _check(load().pqmc_measure(self._h, chain, C.byref(o)), self._h)
        return o.as_dict()

    def dims(self, chain=0):
        d = (C.c_int * 7)()
        _check(load().pqmc_get_dims(self._h, chain, d), self._h)
        return dict(zip(("N", "N_up", "N_dn", "Ltau", "n_stab", "delay_k", "n_fields"), list(d)))

    def measurements(self, chain=0, cap=1 << 16):
        out = np.zeros((cap, RECORD))
        n = C.c_long(cap)
        _check(load().pqmc_get_measurements(self._h, chain, _dptr(out), C.byref(n)), self._h)
        return out[: n.value]

    def last_records(self, out=None):
        """Latest record of every chain (n_chains x RECORD), one device-to-host copy."""
        if out is None:
            out = np.zeros((self.n_chains, RECORD))
        _check(load().pqmc_get_last_records(self._h, _dptr(out)), self._h)
        return out

    def device_bytes(self):
        return int(load().pqmc_device_bytes(self._h))

    def upload_bytes(self):
        return int(load().pqmc_upload_bytes(self._h))

    def green(self, chain=0, spin=0):
        N = self.dims(chain)["N"]
        out = np.zeros((N, N))
        _check(load().pqmc_get_green(self._h, chain, spin, _dptr(out)), self._h)
        return out

    def green_at(self, b, chain=0, spin=0):
        """G at the stabilisation point tau = b * n_stab, recomputed from the
        chain's current fields (the chain's own state is left unchanged)."""
        N = self.dims(chain)["N"]
        out = np.zeros((N, N))
        _check(load().pqmc_get_green_at(self._h, chain, spin, b, _dptr(out)), self._h)
        return out

    def checkpoint(self):
        """The state of every chain and the sweep index, as bytes."""
        n = C.c_size_t(0)
        _check(load().pqmc_checkpoint(self._h, None, C.byref(n)), self._h)
        buf = (C.c_ubyte * n.value)()
        _check(load().pqmc_checkpoint(self._h, buf, C.byref(n)), self._h)
        return bytes(buf)[: n.value]

    def restore(self, data):
        """Load a checkpoint taken from a context with the same specs and options."""
        buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
        _check(load().pqmc_restore(self._h, buf, len(data)), self._h)

    def weight(self, chain=0):
        out = np.zeros(4)
        _check(load().pqmc_get_weight(self._h, chain, _dptr(out)), self._h)
        return out

    def fields(self, chain=0):
        d = self.dims(chain)
        out = np.zeros((d["Ltau"] + 2, d["n_fields"]), dtype=np.int8)
        _check(load().pqmc_get_fields(self._h, chain, out.ctypes.data_as(C.POINTER(C.c_int8))), self._h)
        return out

    def set_fields(self, fields, chain=0):
        f = np.ascontiguousarray(fields, dtype=np.int8)
        _check(load().pqmc_set_fields(self._h, chain, f.ctypes.data_as(C.POINTER(C.c_int8))), self._h)

    def accept_log(self, n, chain=0):
        out = np.zeros(n, dtype=np.uint8)
        _check(load().pqmc_get_accept_log(self._h, chain, out.ctypes.data_as(C.POINTER(C.c_uint8)), n), self._h)
        return out

    def stab_errors(self, chain=0, cap=4096):
        out = np.zeros(cap)
        n = C.c_long(cap)
        _check(load().pqmc_get_stab_errors(self._h, chain, _dptr(out), C.byref(n)), self._h)
        return out[: n.value]

    PHASES = ("flip", "flush", "wrap", "stack", "qr", "refresh", "measure", "total", "qr_form", "overlap", "lu",
              "assemble", "gj_pivot", "gj_elim", "gj_tail", "flush_vec")

    def phase_cycles(self, chain=0):
        out = (C.c_longlong * 16)()
        _check(load().pqmc_get_phase_cycles(self._h, chain, out), self._h)
        return dict(zip(self.PHASES, list(out)))

    def write_run_log(self, path):
        """pqmc_write_run_log: append one JSON line per chain to `path`."""
        _check(load().pqmc_write_run_log(self._h, str(path).encode()), self._h)

    def launch_count(self):
        return int(load().pqmc_launch_count(self._h))

    def launch(self):
        """(delay_k, cta_threads, CTAs per SM, resident shared-memory bytes per chain)."""
        out = (C.c_int * 4)()
        _check(load().pqmc_get_launch(self._h, out), self._h)
        return dict(zip(("delay_k", "cta_threads", "ctas_per_sm", "resident_bytes"), list(out)))

    def inject_error(self, code, chain=0):
        """Test hook: mark a chain failed with ENAN or ESTAB from the host."""
        _check(load().pqmc_inject_error(self._h, chain, code), self._h)


def host_model(spec, spin=0):
    """(K, e^{-dtau K}, P_spin, gap) from the library's host model set-up."""
    lib = load()
    N = spec.n_sites
    ns = (N // 2 if spec.n_up < 0 else spec.n_up) if spin == 0 else (N // 2 if spec.n_dn < 0 else spec.n_dn)
    K = np.zeros((N, N))
    E = np.zeros((N, N))
    P = np.zeros((N, ns))
    gap = C.c_double()
    lat = lattice_of(spec)
    tr = trial_of(spec)
    _check(lib.pqmc_host_model(C.byref(lat), spec.dtau, C.byref(tr), spin, _dptr(K), _dptr(E), _dptr(P),
                               C.byref(gap)))
    return K, E, P, gap.value


def host_eigh(A):
    lib = load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    _check(lib.pqmc_host_eigh(n, _dptr(A), _dptr(w), _dptr(V)))
    return w, V


def autotune(specs, prec=FP64, n_stab=10, delay_k=0, cta_threads=0, dense_chains=0, seed=1):
    """pqmc_autotune: the fastest (delay_k, cta_threads) for the batch, with
    every candidate's time on the proxy batch."""
    lib = load()
    specs = list(specs)
    arr = (ChainSpec * len(specs))(*[chain_spec_of(s) for s in specs])
    opts = Opts(n_stab, delay_k, prec, seed, len(specs), 0, 0, 0, None, cta_threads, dense_chains, 0, 0)
    t = Tune()
    _check(lib.pqmc_autotune(len(specs), arr, C.byref(opts), C.byref(t)))
    return t.as_dict()


PROBE_KEYS = ("fp64_fma_tflops", "fp64_dmma_tflops", "fp32_fma_tflops", "fp64_fma_latency_cycles",
              "fp64_div_latency_cycles", "fp64_sqrt_latency_cycles", "fp64_warp_instr_cycles_1_lane",
              "fp64_warp_instr_cycles_8_lanes", "fp64_warp_instr_cycles_16_lanes", "fp64_warp_instr_cycles_32_lanes",
              "sms", "sm_clock_mhz", "fp64_fma_dmma_mix_tflops", "fp64_fma_dmma_mix_time_ratio")


def probe_pipes():
    """pqmc_probe_pipes: FP64 / DMMA / FP32 throughput and FP64 latencies of the current GPU."""
    out = (C.c_double * 14)()
    _check(load().pqmc_probe_pipes(out))
    return dict(zip(PROBE_KEYS, list(out)))


def test_tc_gemm(M, N, K, d_A, trans_a, d_B, d_C, stream=None):
    """pqmc_test_tc_gemm: device pointers (ints); C = A B by the tensor-core split-BF16 product."""
    _check(load().pqmc_test_tc_gemm(M, N, K, C.c_void_p(d_A), 1 if trans_a else 0, C.c_void_p(d_B),
                                    C.c_void_p(d_C), C.c_void_p(stream) if stream else None))


def host_jackknife(sO, s):
    """(mean, err) of sum(sO)/sum(s) with the library's delete-one-group
    jackknife over the groups whose sums are sO[g], s[g]."""
    sO = np.ascontiguousarray(sO, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    mean, err = C.c_double(), C.c_double()
    _check(load().pqmc_host_jackknife(len(s), _dptr(sO), _dptr(s), C.byref(mean), C.byref(err)))
    return mean.value, err.value


def green_noalloc(spec, n_stab, d_fields, d_G, d_logw, stream=None):
    """pqmc_green_noalloc: device pointers (ints) in and out; no device allocation."""
    cs = chain_spec_of(spec)
    _check(load().pqmc_green_noalloc(C.byref(cs), n_stab, C.c_void_p(d_fields), C.c_void_p(d_G),
                                     C.c_void_p(d_logw), C.c_void_p(stream) if stream else None))
