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


class PcConfig(C.Structure):
    _fields_ = [("eps", C.c_double), ("chi_max", C.c_int32), ("tau", C.c_double),
                ("max_unswap_iter", C.c_int32), ("accept_equal", C.c_int32), ("unswap_mode", C.c_int32),
                ("jacobi_max_sweeps", C.c_int32), ("device", C.c_int32), ("fp32_precondition", C.c_int32)]


class PcStats(C.Structure):
    _fields_ = [("n_updates", C.c_int64), ("n_trials", C.c_int64), ("n_accepted", C.c_int64),
                ("n_stages", C.c_int64), ("n_waves", C.c_int64), ("final_size", C.c_int64),
                ("max_chi", C.c_int32), ("stalled", C.c_int32), ("max_sweeps", C.c_int32), ("fallbacks", C.c_int32),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


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
           "pc_restore", "pc_get_stream", "pc_factorise_noalloc"]


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
        "pc_set_cursors": ([vp, i64, i64], i32),
        "pc_snapshot": ([vp], i32),
        "pc_restore": ([vp], i32),
        "pc_get_stream": ([vp, _p(vp)], i32),
        "pc_factorise_noalloc": ([vp, i32, i32, dbl, i32, vp, vp, _p(i32), vp], i32),
        "pc_reset_kernel_timers": ([vp, i32], i32),
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
        """(launches, ms, flops) per kernel class: merge+gate, Jacobi, truncate, split, other."""
        la = np.zeros(5, dtype=np.int64)
        ms = np.zeros(5)
        fl = np.zeros(5)
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
