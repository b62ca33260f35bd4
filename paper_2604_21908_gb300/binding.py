"""Thin ctypes binding of libpeaked_mpo.so (argument marshalling only).

Every function here calls straight into the C ABI declared in include/peaked_mpo.h; all
computation happens in the library's CUDA kernels.  There is no fallback: if the shared
library is missing or fails to load, load() raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpeaked_mpo.so")

PC_OK = 0
STATUS_NAMES = {0: "PC_OK", -1: "PC_ERR_INVALID_ARG", -2: "PC_ERR_NONUNITARY", -3: "PC_ERR_OOM",
                -4: "PC_ERR_NOCONVERGE", -5: "PC_ERR_TIMEOUT", -6: "PC_ERR_NOT_PEAKED", -7: "PC_ERR_CUDA",
                -8: "PC_ERR_STATE", 1: "PC_WARN_STALLED"}
UNSWAP_PARALLEL, UNSWAP_SEQUENTIAL, UNSWAP_OFF = 0, 1, 2
PRECISION_FP64, PRECISION_TF32X3 = 0, 1
SIDE_ALTERNATE, SIDE_ADAPTIVE = 0, 1


class PcConfig(C.Structure):
    _fields_ = [("eps", C.c_double), ("chi_max", C.c_int32), ("tau", C.c_double),
                ("max_unswap_iter", C.c_int32), ("accept_equal", C.c_int32), ("unswap_mode", C.c_int32),
                ("jacobi_max_sweeps", C.c_int32), ("device", C.c_int32), ("fp32_precondition", C.c_int32),
                ("precision", C.c_int32), ("precondition_sweeps", C.c_int32), ("side_mode", C.c_int32),
                ("certify_trials", C.c_int32), ("deflate", C.c_int32), ("fp32_dead_rel", C.c_double),
                ("recanonicalise", C.c_int32), ("pad_", C.c_int32)]


class PcStats(C.Structure):
    _fields_ = [("n_updates", C.c_int64), ("n_trials", C.c_int64), ("n_accepted", C.c_int64),
                ("n_stages", C.c_int64), ("n_waves", C.c_int64), ("final_size", C.c_int64),
                ("max_chi", C.c_int32), ("stalled", C.c_int32), ("max_sweeps", C.c_int32), ("fallbacks", C.c_int32),
                ("seconds", C.c_double), ("max_sweeps_fp32", C.c_int32), ("pad_", C.c_int32),
                ("n_trials_certified", C.c_int64), ("n_deflated", C.c_int64), ("n_full", C.c_int64),
                ("n_recanon", C.c_int64), ("alg_flops", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


class PcTraceRecord(C.Structure):
    _fields_ = [("stage", C.c_int32), ("phase", C.c_int32), ("gates", C.c_int64), ("size", C.c_int64),
                ("max_chi", C.c_int32), ("accepted", C.c_int32), ("seconds", C.c_double)]


class PcServerConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_resident", C.c_int32), ("memory_budget", C.c_int64),
                ("max_tasks", C.c_int32), ("arena_bytes", C.c_int64)]


class PcRequest(C.Structure):
    _fields_ = [("cfg", PcConfig), ("n_qubits", C.c_int32), ("n_gates", C.c_int64), ("pairs", C.c_void_p),
                ("mats", C.c_void_p), ("split_index", C.c_int64), ("n_oneq", C.c_int64),
                ("oneq_qubits", C.c_void_p), ("oneq_mats", C.c_void_p), ("n_samples", C.c_int64),
                ("seed", C.c_uint64)]


class PcResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_qubits", C.c_int32), ("p_peak", C.c_double), ("norm2", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("n_updates", C.c_int64), ("n_trials", C.c_int64), ("n_accepted", C.c_int64),
                ("max_chi", C.c_int32), ("store_bytes", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("resident", C.c_int32), ("max_resident_seen", C.c_int32), ("bytes_resident", C.c_int64),
                ("max_bytes_seen", C.c_int64), ("p50_s", C.c_double), ("p99_s", C.c_double), ("mean_s", C.c_double),
                ("circuits_per_hour", C.c_double), ("launches", C.c_int64), ("tasks", C.c_int64),
                ("max_tasks_per_launch", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_LIB = None

EXPORTS = ["pc_version", "pc_default_config", "pc_create", "pc_destroy", "pc_last_error", "pc_load_gates",
           "pc_destroy_circuit", "pc_contract", "pc_unswap", "pc_extract_peak", "pc_sample", "pc_amplitudes",
           "pc_get_bond_dims", "pc_get_layouts", "pc_get_spectrum", "pc_get_site", "pc_set_state",
           "pc_apply_updates", "pc_plan_routing", "pc_get_plan", "pc_get_unswap_log", "pc_kernel_timers",
           "pc_reset_kernel_timers", "pc_contract_iterations", "pc_get_cursors", "pc_set_cursors", "pc_snapshot",
           "pc_restore", "pc_get_stream", "pc_factorise_noalloc", "pc_get_stats", "pc_get_trace", "pc_checkpoint_write", "pc_checkpoint_read", "pc_batch_create", "pc_batch_destroy",
           "pc_batch_attach", "pc_batch_detach", "pc_batch_contract", "pc_batch_counters", "pc_batch_set_timing",
           "pc_projected_bytes", "pc_server_create", "pc_server_submit", "pc_server_wait", "pc_server_get_stats",
           "pc_server_clock", "pc_server_destroy", "pc_measure_alu_peaks", "pc_autotune", "pc_load_tuning"]


def _p(t):
    return C.POINTER(t)


def load(path: str = LIB_PATH):
    """Loads the library (building it first if the source is newer) and declares signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = C.CDLL(path)
    i32, i64, u64, dbl = C.c_int32, C.c_int64, C.c_uint64, C.c_double
    vp = C.c_void_p
    sig = {
        "pc_version": ([], C.c_char_p),
        "pc_default_config": ([_p(PcConfig)], None),
        "pc_create": ([_p(PcConfig), _p(vp)], i32),
        "pc_destroy": ([vp], i32),
        "pc_last_error": ([vp], C.c_char_p),
        "pc_load_gates": ([vp, i32, i64, vp, vp, i64, i64, vp, vp, _p(vp)], i32),
        "pc_destroy_circuit": ([vp], i32),
        "pc_contract": ([vp, _p(PcStats)], i32),
        "pc_unswap": ([vp, _p(i32)], i32),
        "pc_extract_peak": ([vp, i64, vp, _p(dbl), _p(dbl)], i32),
        "pc_sample": ([vp, i64, u64, vp], i32),
        "pc_amplitudes": ([vp, i64, vp, vp], i32),
        "pc_get_bond_dims": ([vp, vp], i32),
        "pc_get_layouts": ([vp, vp, vp], i32),
        "pc_get_spectrum": ([vp, i32, i32, vp, _p(i32)], i32),
        "pc_get_site": ([vp, i32, i64, vp, vp], i32),
        "pc_set_state": ([vp, vp, vp, vp], i32),
        "pc_apply_updates": ([vp, i32, vp, vp, vp], i32),
        "pc_plan_routing": ([i32, i64, vp, i64, i64, vp, _p(i64)], i32),
        "pc_get_plan": ([vp, i64, vp, _p(i64)], i32),
        "pc_get_unswap_log": ([vp, i64, vp, _p(i64)], i32),
        "pc_kernel_timers": ([vp, vp, vp, vp], i32),
        "pc_contract_iterations": ([vp, i32, _p(PcStats), _p(i32)], i32),
        "pc_get_cursors": ([vp, _p(i64), _p(i64)], i32),
        "pc_get_stats": ([vp, _p(PcStats)], i32),
        "pc_get_trace": ([vp, i64, vp, _p(i64)], i32),
        "pc_checkpoint_write": ([vp, C.c_char_p], i32),
        "pc_checkpoint_read": ([vp, C.c_char_p], i32),
        "pc_set_cursors": ([vp, i64, i64], i32),
        "pc_snapshot": ([vp], i32),
        "pc_restore": ([vp], i32),
        "pc_get_stream": ([vp, _p(vp)], i32),
        "pc_factorise_noalloc": ([vp, i32, i32, dbl, i32, vp, vp, _p(i32), vp], i32),
        "pc_reset_kernel_timers": ([vp, i32], i32),
        "pc_batch_create": ([vp, i32, i64, _p(vp)], i32),
        "pc_batch_destroy": ([vp], i32),
        "pc_batch_attach": ([vp, vp], i32),
        "pc_batch_detach": ([vp, vp], i32),
        "pc_batch_contract": ([vp, i32, vp, vp, vp], i32),
        "pc_batch_counters": ([vp, _p(i64), _p(i64), _p(i32), vp, vp], i32),
        "pc_batch_set_timing": ([vp, i32], i32),
        "pc_projected_bytes": ([i32, i32, i64], i64),
        "pc_measure_alu_peaks": ([i32, _p(dbl), _p(dbl)], i32),
        "pc_autotune": ([i32, i32, vp, vp, C.c_char_p, vp], i32),
        "pc_load_tuning": ([C.c_char_p], i32),
        "pc_server_create": ([_p(PcServerConfig), _p(vp)], i32),
        "pc_server_submit": ([vp, _p(PcRequest), _p(i64)], i32),
        "pc_server_wait": ([vp, i64, dbl, _p(PcResult), vp, vp], i32),
        "pc_server_get_stats": ([vp, _p(PcServerStats)], i32),
        "pc_server_clock": ([vp], dbl),
        "pc_server_destroy": ([vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_config(**kw) -> PcConfig:
    lib = load()
    cfg = PcConfig()
    lib.pc_default_config(C.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def measure_alu_peaks(device: int = 0) -> tuple[float, float]:
    """pc_measure_alu_peaks: (FP64, FP32) FMA-chain TFLOP/s of the device."""
    lib = load()
    a, b = C.c_double(0), C.c_double(0)
    st = lib.pc_measure_alu_peaks(device, C.byref(a), C.byref(b))
    if st != PC_OK:
        raise PcError(st, "pc_measure_alu_peaks")
    return a.value, b.value


def autotune(shapes, path: str | None = None, device: int = 0) -> np.ndarray:
    """pc_autotune over (row length, matrices per launch) shapes; returns ms[n][3] for group
    widths 1, 2, 4 and installs the fastest width per shape."""
    lib = load()
    lens = np.ascontiguousarray([s[0] for s in shapes], dtype=np.int32)
    bats = np.ascontiguousarray([s[1] for s in shapes], dtype=np.int32)
    ms = np.zeros((len(shapes), 3))
    st = lib.pc_autotune(device, len(shapes), _ptr(lens), _ptr(bats), path.encode() if path else None, _ptr(ms))
    if st != PC_OK:
        raise PcError(st, "pc_autotune")
    return ms


def load_tuning(path: str) -> None:
    st = load().pc_load_tuning(path.encode())
    if st != PC_OK:
        raise PcError(st, "pc_load_tuning")


def plan_routing(n_qubits: int, pairs: np.ndarray, split_index: int) -> np.ndarray:
    """pc_plan_routing: (side, bond, kind, gate) records of the router with unswapping off."""
    lib = load()
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    n_rec = C.c_int64(0)
    st = lib.pc_plan_routing(n_qubits, pairs.shape[0], _ptr(pairs), split_index, 0, None, C.byref(n_rec))
    if st != PC_OK:
        raise PcError(st, "pc_plan_routing")
    rec = np.zeros((max(n_rec.value, 1), 4), dtype=np.int32)
    st = lib.pc_plan_routing(n_qubits, pairs.shape[0], _ptr(pairs), split_index, rec.shape[0], _ptr(rec),
                             C.byref(n_rec))
    if st != PC_OK:
        raise PcError(st, "pc_plan_routing")
    return rec[: n_rec.value]


def factorise_noalloc(x_ptr: int, m: int, n: int, eps: float, chi_max: int, s_ptr: int, vh_ptr: int,
                      stream: int = 0) -> int:
    """pc_factorise_noalloc on caller-owned device buffers (addresses as integers); returns
    the number of kept values."""
    lib = load()
    k = C.c_int32(0)
    st = lib.pc_factorise_noalloc(C.c_void_p(x_ptr), m, n, eps, chi_max, C.c_void_p(s_ptr), C.c_void_p(vh_ptr),
                                  C.byref(k), C.c_void_p(stream) if stream else None)
    if st != PC_OK:
        raise PcError(st, "pc_factorise_noalloc")
    return k.value


class Context:
    def __init__(self, **cfg_kw):
        self.lib = load()
        self.cfg = default_config(**cfg_kw)
        h = C.c_void_p()
        st = self.lib.pc_create(C.byref(self.cfg), C.byref(h))
        if st != PC_OK:
            raise PcError(st, "pc_create")
        self.h = h

    def check(self, st, what):
        if st < 0:
            raise PcError(st, f"{what}: {self.lib.pc_last_error(self.h).decode()}")
        return st

    def load_gates(self, n_qubits, pairs, mats, split_index=-1, oneq_qubits=None, oneq_mats=None):
        """pc_load_gates.  mats: complex [G,4,4] or float64 [G,4,4,2]."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        mats = np.asarray(mats)
        if np.iscomplexobj(mats):
            mats = np.stack([mats.real, mats.imag], axis=-1)
        mats = np.ascontiguousarray(mats, dtype=np.float64)
        if oneq_qubits is None or len(oneq_qubits) == 0:
            oq = np.zeros(0, np.int32)
            om = np.zeros((0, 2, 2, 2))
        else:
            oq = np.ascontiguousarray(oneq_qubits, dtype=np.int32)
            om = np.asarray(oneq_mats)
            if np.iscomplexobj(om):
                om = np.stack([om.real, om.imag], axis=-1)
            om = np.ascontiguousarray(om, dtype=np.float64)
        h = C.c_void_p()
        st = self.lib.pc_load_gates(self.h, n_qubits, pairs.shape[0], _ptr(pairs), _ptr(mats), split_index,
                                    oq.shape[0], _ptr(oq), _ptr(om), C.byref(h))
        self.check(st, "pc_load_gates")
        return Circuit(self, h, n_qubits)

    def load_circuit(self, circ):
        """Loads a workloads.Circuit."""
        return self.load_gates(circ.n_qubits, circ.pairs, circ.mats, circ.split_index, circ.oneq_qubits,
                               circ.oneq_mats)

    def close(self):
        if self.h:
            self.lib.pc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Circuit:
    def __init__(self, ctx: Context, h, n):
        self.ctx, self.h, self.n = ctx, h, n
        self.lib = ctx.lib

    def _chk(self, st, what):
        return self.ctx.check(st, what)

    def contract(self) -> dict:
        stats = PcStats()
        st = self.lib.pc_contract(self.h, C.byref(stats))
        self._chk(st, "pc_contract")
        d = stats.as_dict()
        d["status"] = st
        return d

    def contract_iterations(self, max_iterations: int):
        stats = PcStats()
        done = C.c_int32(0)
        self._chk(self.lib.pc_contract_iterations(self.h, max_iterations, C.byref(stats), C.byref(done)),
                  "pc_contract_iterations")
        d = stats.as_dict()
        d["done"] = bool(done.value)
        return d

    def stats(self) -> dict:
        """pc_get_stats: counters since the last contraction call began."""
        out = PcStats()
        self._chk(self.lib.pc_get_stats(self.h, C.byref(out)), "pc_get_stats")
        return out.as_dict()

    def trace(self) -> list[dict]:
        """pc_get_trace: (stage, phase, gates, size, max_chi, accepted, seconds) records."""
        n = C.c_int64(0)
        self._chk(self.lib.pc_get_trace(self.h, 0, None, C.byref(n)), "pc_get_trace")
        recs = (PcTraceRecord * max(n.value, 1))()
        self._chk(self.lib.pc_get_trace(self.h, n.value, C.cast(recs, C.c_void_p), C.byref(n)), "pc_get_trace")
        return [{f: getattr(recs[k], f) for f, _ in PcTraceRecord._fields_} for k in range(n.value)]

    def cursors(self):
        a, b = C.c_int64(0), C.c_int64(0)
        self._chk(self.lib.pc_get_cursors(self.h, C.byref(a), C.byref(b)), "pc_get_cursors")
        return a.value, b.value

    def set_cursors(self, left: int, right: int):
        self._chk(self.lib.pc_set_cursors(self.h, left, right), "pc_set_cursors")

    def stream_handle(self) -> int:
        """The circuit's cudaStream_t as an integer (for torch.cuda.ExternalStream)."""
        h = C.c_void_p()
        self._chk(self.lib.pc_get_stream(self.h, C.byref(h)), "pc_get_stream")
        return h.value or 0

    def checkpoint_write(self, path: str):
        self._chk(self.lib.pc_checkpoint_write(self.h, os.fsencode(path)), "pc_checkpoint_write")

    def checkpoint_read(self, path: str):
        self._chk(self.lib.pc_checkpoint_read(self.h, os.fsencode(path)), "pc_checkpoint_read")

    def snapshot(self):
        self._chk(self.lib.pc_snapshot(self.h), "pc_snapshot")

    def restore(self):
        self._chk(self.lib.pc_restore(self.h), "pc_restore")

    def unswap(self) -> int:
        acc = C.c_int32(0)
        self._chk(self.lib.pc_unswap(self.h, C.byref(acc)), "pc_unswap")
        return acc.value

    def extract_peak(self, max_expansions=100000):
        bits = np.zeros(self.n, dtype=np.uint8)
        p = C.c_double(0)
        z = C.c_double(0)
        self._chk(self.lib.pc_extract_peak(self.h, max_expansions, _ptr(bits), C.byref(p), C.byref(z)),
                  "pc_extract_peak")
        return bits, p.value, z.value

    def sample(self, n_samples, seed):
        bits = np.zeros((n_samples, self.n), dtype=np.uint8)
        self._chk(self.lib.pc_sample(self.h, n_samples, seed, _ptr(bits)), "pc_sample")
        return bits

    def amplitudes(self, bits):
        bits = np.ascontiguousarray(bits, dtype=np.uint8).reshape(-1, self.n)
        amp = np.zeros((bits.shape[0], 2))
        self._chk(self.lib.pc_amplitudes(self.h, bits.shape[0], _ptr(bits), _ptr(amp)), "pc_amplitudes")
        return amp[:, 0] + 1j * amp[:, 1]

    def bond_dims(self):
        chi = np.zeros(self.n - 1, dtype=np.int32)
        self._chk(self.lib.pc_get_bond_dims(self.h, _ptr(chi)), "pc_get_bond_dims")
        return chi

    def layouts(self):
        a = np.zeros(self.n, dtype=np.int32)
        b = np.zeros(self.n, dtype=np.int32)
        self._chk(self.lib.pc_get_layouts(self.h, _ptr(a), _ptr(b)), "pc_get_layouts")
        return a, b

    def spectrum(self, bond):
        ln = C.c_int32(0)
        self._chk(self.lib.pc_get_spectrum(self.h, bond, 0, None, C.byref(ln)), "pc_get_spectrum")
        s = np.zeros(ln.value)
        self._chk(self.lib.pc_get_spectrum(self.h, bond, ln.value, _ptr(s), C.byref(ln)), "pc_get_spectrum")
        return s

    def site(self, j):
        dims = np.zeros(2, dtype=np.int32)
        self._chk(self.lib.pc_get_site(self.h, j, 0, None, _ptr(dims)), "pc_get_site")
        out = np.zeros((dims[0], 4, dims[1], 2))
        self._chk(self.lib.pc_get_site(self.h, j, out.size // 2, _ptr(out), _ptr(dims)), "pc_get_site")
        return out[..., 0] + 1j * out[..., 1]

    def set_state(self, B, lam):
        chi = np.array([1] + [b.shape[2] for b in B[:-1]] + [1], dtype=np.int32)
        sites = np.concatenate([np.stack([b.real, b.imag], -1).ravel() for b in B]).astype(np.float64)
        lm = np.concatenate([np.asarray(x, np.float64).ravel() for x in lam]) if lam else np.zeros(0)
        self._chk(self.lib.pc_set_state(self.h, _ptr(chi), _ptr(sites), _ptr(lm)), "pc_set_state")

    def apply_updates(self, bonds, ops):
        bonds = np.ascontiguousarray(bonds, dtype=np.int32)
        ops = np.asarray(ops).reshape(len(bonds), 16, 16)
        o = np.ascontiguousarray(np.stack([ops.real, ops.imag], -1), dtype=np.float64)
        chi = np.zeros(len(bonds), dtype=np.int32)
        self._chk(self.lib.pc_apply_updates(self.h, len(bonds), _ptr(bonds), _ptr(o), _ptr(chi)), "pc_apply_updates")
        return chi

    def plan(self):
        n = C.c_int64(0)
        self._chk(self.lib.pc_get_plan(self.h, 0, None, C.byref(n)), "pc_get_plan")
        rec = np.zeros((max(n.value, 1), 5), dtype=np.int32)
        self._chk(self.lib.pc_get_plan(self.h, rec.shape[0], _ptr(rec), C.byref(n)), "pc_get_plan")
        return rec[: n.value]

    def unswap_log(self):
        n = C.c_int64(0)
        self._chk(self.lib.pc_get_unswap_log(self.h, 0, None, C.byref(n)), "pc_get_unswap_log")
        rec = np.zeros((max(n.value, 1), 4), dtype=np.int32)
        self._chk(self.lib.pc_get_unswap_log(self.h, rec.shape[0], _ptr(rec), C.byref(n)), "pc_get_unswap_log")
        return rec[: n.value]

    def reset_timers(self, enable=True):
        self._chk(self.lib.pc_reset_kernel_timers(self.h, 1 if enable else 0), "pc_reset_kernel_timers")

    def timers(self):
        """(launches, ms, flops) per kernel class: merge+gate, factorisation, truncate, split,
        other, unswap-trial certificates."""
        la = np.zeros(6, dtype=np.int64)
        ms = np.zeros(6)
        fl = np.zeros(6)
        self._chk(self.lib.pc_kernel_timers(self.h, _ptr(la), _ptr(ms), _ptr(fl)), "pc_kernel_timers")
        return la, ms, fl

    def close(self):
        if self.h:
            self.lib.pc_destroy_circuit(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def projected_bytes(n_qubits: int, chi_max: int, n_samples: int = 0) -> int:
    """pc_projected_bytes: device bytes a served circuit keeps resident (host-only)."""
    return int(load().pc_projected_bytes(n_qubits, chi_max, n_samples))


def _gate_arrays(circ):
    pairs = np.ascontiguousarray(circ.pairs, dtype=np.int32).reshape(-1, 2)
    mats = np.asarray(circ.mats)
    if np.iscomplexobj(mats):
        mats = np.stack([mats.real, mats.imag], axis=-1)
    mats = np.ascontiguousarray(mats, dtype=np.float64).reshape(-1, 4, 4, 2)
    if circ.oneq_qubits is None or len(circ.oneq_qubits) == 0:
        oq = np.zeros(0, np.int32)
        om = np.zeros((0, 2, 2, 2))
    else:
        oq = np.ascontiguousarray(circ.oneq_qubits, dtype=np.int32)
        om = np.asarray(circ.oneq_mats)
        if np.iscomplexobj(om):
            om = np.stack([om.real, om.imag], axis=-1)
        om = np.ascontiguousarray(om, dtype=np.float64)
    return pairs, mats, oq, om


class Batch:
    """pc_batch_*: combined launches of the waves of several circuits."""

    def __init__(self, ctx: Context, max_tasks: int = 256, arena_bytes: int = 0):
        self.ctx, self.lib = ctx, ctx.lib
        h = C.c_void_p()
        ctx.check(self.lib.pc_batch_create(ctx.h, max_tasks, arena_bytes, C.byref(h)), "pc_batch_create")
        self.h = h

    def contract(self, circuits):
        """pc_batch_contract: returns (statuses, list of stats dicts)."""
        n = len(circuits)
        handles = (C.c_void_p * n)(*[c.h for c in circuits])
        statuses = np.zeros(n, dtype=np.int32)
        stats = (PcStats * n)()
        st = self.lib.pc_batch_contract(self.h, n, C.cast(handles, C.c_void_p), _ptr(statuses),
                                        C.cast(stats, C.c_void_p))
        for k, c in enumerate(circuits):
            if statuses[k] < 0:
                c._chk(int(statuses[k]), "pc_batch_contract")
        if st < 0:
            raise PcError(st, "pc_batch_contract")
        return statuses, [s.as_dict() for s in stats]

    def counters(self):
        la, ta = C.c_int64(0), C.c_int64(0)
        mt = C.c_int32(0)
        ms = np.zeros(6)
        fl = np.zeros(6)
        self.lib.pc_batch_counters(self.h, C.byref(la), C.byref(ta), C.byref(mt), _ptr(ms), _ptr(fl))
        return {"launches": la.value, "tasks": ta.value, "max_tasks": mt.value, "ms": ms, "flops": fl}

    def set_timing(self, enable=True):
        self.lib.pc_batch_set_timing(self.h, 1 if enable else 0)

    def close(self):
        if self.h:
            self.lib.pc_batch_destroy(self.h)
            self.h = None


class Server:
    """pc_server_*: request loop with admission by projected device memory and continuous
    batching of every resident circuit's factorisations."""

    def __init__(self, max_resident=8, memory_budget=64 << 30, max_tasks=256, arena_bytes=0, device=0):
        self.lib = load()
        cfg = PcServerConfig(device, max_resident, memory_budget, max_tasks, arena_bytes)
        h = C.c_void_p()
        st = self.lib.pc_server_create(C.byref(cfg), C.byref(h))
        if st != PC_OK:
            raise PcError(st, "pc_server_create")
        self.h = h
        self.n_of = {}
        self.samples_of = {}

    def submit(self, circ, n_samples=0, seed=0, **cfg_kw) -> int:
        pairs, mats, oq, om = _gate_arrays(circ)
        req = PcRequest()
        req.cfg = default_config(**cfg_kw)
        req.n_qubits = circ.n_qubits
        req.n_gates = pairs.shape[0]
        req.pairs = pairs.ctypes.data
        req.mats = mats.ctypes.data
        req.split_index = circ.split_index
        req.n_oneq = oq.shape[0]
        req.oneq_qubits = oq.ctypes.data
        req.oneq_mats = om.ctypes.data
        req.n_samples = n_samples
        req.seed = seed
        t = C.c_int64(0)
        st = self.lib.pc_server_submit(self.h, C.byref(req), C.byref(t))
        if st != PC_OK:
            raise PcError(st, "pc_server_submit")
        self.n_of[t.value] = circ.n_qubits
        self.samples_of[t.value] = n_samples
        return t.value

    def wait(self, ticket, timeout_s=-1.0):
        """(result dict, peak bits, samples or None)."""
        n, S = self.n_of[ticket], self.samples_of[ticket]
        res = PcResult()
        bits = np.zeros(n, dtype=np.uint8)
        samples = np.zeros((S, n), dtype=np.uint8) if S > 0 else None
        st = self.lib.pc_server_wait(self.h, ticket, timeout_s, C.byref(res), _ptr(bits),
                                     _ptr(samples) if samples is not None else None)
        if st != PC_OK:
            raise PcError(st, "pc_server_wait")
        return res.as_dict(), bits, samples

    def stats(self) -> dict:
        out = PcServerStats()
        self.lib.pc_server_get_stats(self.h, C.byref(out))
        return out.as_dict()

    def clock(self) -> float:
        return float(self.lib.pc_server_clock(self.h))

    def close(self):
        if self.h:
            self.lib.pc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
