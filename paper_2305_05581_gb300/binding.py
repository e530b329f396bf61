"""ctypes binding of the C ABI in include/tns.h (argument marshalling only).

Every computation happens inside the shared library; this module converts
Python arguments to pointers and sizes and turns error codes into
exceptions.  Device pointers are plain integers (e.g. ``tensor.data_ptr()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

TNS_FP64, TNS_TF32, TNS_BF16X3 = 0, 1, 2
ERRORS = {-1: "TNS_ERR_ARG", -2: "TNS_ERR_STATE", -3: "TNS_ERR_OOM", -4: "TNS_ERR_NOCONV",
          -5: "TNS_ERR_DEVICE_TIMEOUT", -6: "TNS_ERR_CUDA"}

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_LIB = os.path.join(HERE, "libtns.so")

# every entry point of include/tns.h
SYMBOLS = ["create", "destroy", "last_error", "load_integrals", "mps_init", "mps_define",
           "mps_set_bond", "mps_set_site", "mps_get_bond", "mps_get_site", "build_env",
           "psi_layout", "heff_apply", "heff_diag", "davidson", "sweep", "heff_flops", "step", "psi_guess",
           "heff_diag_noalloc", "env_arena", "heff_adjoint", "sym_eig", "rdm", "set_memory_budget",
           "memory_stats", "heff_apply_part",
           "checkpoint_save", "checkpoint_load",
           "schedule_stats"]


class TnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SweepOpts(C.Structure):
    _fields_ = [("nsweeps", C.c_int), ("D", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("precision", C.c_int), ("cutoff", C.c_double), ("verbose", C.c_int), ("block", C.c_int)]


class SweepStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_discarded", C.c_double), ("matvecs", C.c_longlong),
                ("heff_flops", C.c_double), ("heff_seconds", C.c_double), ("env_seconds", C.c_double),
                ("svd_seconds", C.c_double), ("seconds", C.c_double), ("steps", C.c_int),
                ("max_bond", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("discarded", C.c_double), ("iters", C.c_int), ("converged", C.c_int),
                ("heff_flops", C.c_double), ("heff_seconds", C.c_double), ("env_seconds", C.c_double),
                ("svd_seconds", C.c_double), ("seconds", C.c_double), ("length", C.c_longlong),
                ("bond_dim", C.c_int), ("kernel_launches", C.c_longlong), ("exact_products", C.c_int),
                ("exact_seconds", C.c_double), ("env_flops", C.c_double), ("env_bytes", C.c_double)]


class SchedStats(C.Structure):
    _fields_ = [("tuned", C.c_longlong), ("cache_hits", C.c_longlong), ("runs", (C.c_longlong * 4) * 3)]

    def as_dict(self):
        names = ["fp64", "tf32", "bf16x3"]
        return {"tuned": int(self.tuned), "cache_hits": int(self.cache_hits),
                "runs": {names[p]: [int(self.runs[p][v]) for v in range(4)] for p in range(3)}}


class MemStats(C.Structure):
    _fields_ = [("device_used", C.c_longlong), ("device_peak", C.c_longlong), ("device_limit", C.c_longlong),
                ("host_used", C.c_longlong), ("host_peak", C.c_longlong), ("staged", C.c_longlong),
                ("restored", C.c_longlong), ("dropped", C.c_longlong), ("built", C.c_longlong),
                ("last_plan", C.c_longlong)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


_LIBS = {}


def load_library(path: str = DEFAULT_LIB, prefix: str = "tns_"):
    key = (path, prefix)
    if key in _LIBS:
        return _LIBS[key]
    if not os.path.exists(path):
        raise OSError(f"shared library {path} not found: build it first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    f = lambda n: getattr(lib, prefix + n)
    vp, ip, dp, llp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_longlong)
    sig = {
        "create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
        "destroy": (None, [vp]),
        "last_error": (C.c_char_p, [vp]),
        "load_integrals": (C.c_int, [vp, C.c_int, dp, dp, C.c_double]),
        "mps_init": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong]),
        "mps_define": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int]),
        "mps_set_bond": (C.c_int, [vp, C.c_int, C.c_int, ip, ip]),
        "mps_set_site": (C.c_int, [vp, C.c_int, dp, C.c_longlong]),
        "mps_get_bond": (C.c_int, [vp, C.c_int, ip, ip, ip, C.c_int]),
        "mps_get_site": (C.c_int, [vp, C.c_int, dp, C.c_longlong, llp]),
        "build_env": (C.c_int, [vp, C.c_int]),
        "psi_layout": (C.c_int, [vp, C.c_int, ip, C.POINTER(llp), llp]),
        "heff_apply": (C.c_int, [vp, C.c_int, vp, vp, C.c_int, C.c_int]),
        "heff_diag": (C.c_int, [vp, C.c_int, vp]),
        "heff_apply_part": (C.c_int, [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int]),
        "davidson": (C.c_int, [vp, C.c_int, vp, C.c_double, C.c_int, C.c_int, dp, ip]),
        "sweep": (C.c_int, [vp, C.POINTER(SweepOpts), dp, C.POINTER(SweepStats)]),
        "heff_flops": (C.c_int, [vp, C.c_int, dp, llp]),
        "step": (C.c_int, [vp, C.c_int, C.c_int, C.POINTER(SweepOpts), vp, vp, C.POINTER(StepStats)]),
        "psi_guess": (C.c_int, [vp, C.c_int, vp, llp]),
        "heff_diag_noalloc": (C.c_int, [vp, C.c_int, vp]),
        "env_arena": (C.c_int, [vp, C.c_int, C.c_int, C.POINTER(vp), llp]),
        "heff_adjoint": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, vp]),
        "sym_eig": (C.c_int, [vp, C.c_int, ip, vp, vp, vp]),
        "rdm": (C.c_int, [vp, C.c_int, vp, dp, dp]),
        "set_memory_budget": (C.c_int, [vp, C.c_longlong, C.c_longlong]),
        "checkpoint_save": (C.c_int, [vp, C.c_char_p, C.c_int, C.c_int]),
        "schedule_stats": (C.c_int, [vp, C.POINTER(SchedStats)]),
        "checkpoint_load": (C.c_int, [vp, C.c_char_p, ip, ip]),
        "memory_stats": (C.c_int, [vp, C.POINTER(MemStats), C.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = f(name)
        fn.restype = res
        fn.argtypes = args
    _LIBS[key] = (lib, prefix)
    return _LIBS[key]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Context:
    """One engine context (one device, one stream)."""

    def __init__(self, device: int = 0, stream: int | None = None, path: str = DEFAULT_LIB,
                 prefix: str = "tns_"):
        self._lib, self._pfx = load_library(path, prefix)
        h = C.c_void_p()
        rc = self._fn("create")(C.byref(h), device, C.c_void_p(stream) if stream else None)
        if rc != 0:
            raise TnsError(rc, "create failed")
        self._h = h

    def _fn(self, name):
        return getattr(self._lib, self._pfx + name)

    def _check(self, rc):
        if rc != 0:
            msg = self._fn("last_error")(self._h).decode()
            raise TnsError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._fn("destroy")(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- problem definition -------------------------------------------------
    def load_integrals(self, h, v, e_core: float = 0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        self._check(self._fn("load_integrals")(self._h, h.shape[0], _dptr(h), _dptr(v), float(e_core)))

    def mps_init(self, N, n_elec, two_sz, D, seed=0):
        self._check(self._fn("mps_init")(self._h, N, n_elec, two_sz, D, seed))

    def mps_import(self, N, n_elec, two_sz, D, bonds, sites):
        """bonds[b] = [((n, 2sz), dim)], sites[b] = {(q_l, s): array} (see synth)."""
        self._check(self._fn("mps_define")(self._h, N, n_elec, two_sz, D))
        for b, bond in enumerate(bonds):
            sec = np.array([x for (q, d) in bond for x in q], dtype=np.int32)
            dims = np.array([d for (q, d) in bond], dtype=np.int32)
            self._check(self._fn("mps_set_bond")(self._h, b, len(bond), sec.ctypes.data_as(C.POINTER(C.c_int)),
                                                  dims.ctypes.data_as(C.POINTER(C.c_int))))
        qn = [(0, 0), (1, 1), (1, -1), (2, 0)]
        for b in range(N):
            right = {q for q, _ in bonds[b + 1]}
            parts = []
            for ql, dl in bonds[b]:
                for s in range(4):
                    qr = (ql[0] + qn[s][0], ql[1] + qn[s][1])
                    if qr in right:
                        parts.append(np.ascontiguousarray(sites[b][(ql, s)], dtype=np.float64).ravel())
            data = np.concatenate(parts) if parts else np.zeros(0)
            self._check(self._fn("mps_set_site")(self._h, b, _dptr(data), data.size))

    def get_bond(self, b):
        n = C.c_int()
        self._check(self._fn("mps_get_bond")(self._h, b, C.byref(n), None, None, 0))
        sec = np.zeros(2 * n.value, dtype=np.int32)
        dims = np.zeros(n.value, dtype=np.int32)
        self._check(self._fn("mps_get_bond")(self._h, b, C.byref(n), sec.ctypes.data_as(C.POINTER(C.c_int)),
                                              dims.ctypes.data_as(C.POINTER(C.c_int)), n.value))
        return [((int(sec[2 * i]), int(sec[2 * i + 1])), int(dims[i])) for i in range(n.value)]

    def get_site(self, b):
        n = C.c_longlong()
        self._check(self._fn("mps_get_site")(self._h, b, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        self._check(self._fn("mps_get_site")(self._h, b, _dptr(out), n.value, None))
        return out

    # -- two-site step --------------------------------------------------------
    def build_env(self, site):
        self._check(self._fn("build_env")(self._h, site))

    def psi_layout(self, site):
        nb = C.c_int()
        p = C.POINTER(C.c_longlong)()
        ln = C.c_longlong()
        self._check(self._fn("psi_layout")(self._h, site, C.byref(nb), C.byref(p), C.byref(ln)))
        desc = np.ctypeslib.as_array(p, shape=(nb.value * 9,)).reshape(nb.value, 9).copy()
        return desc, ln.value

    def heff_apply_ptr(self, site, x_ptr: int, y_ptr: int, nvec: int = 1, precision: int = TNS_FP64):
        self._check(self._fn("heff_apply")(self._h, site, C.c_void_p(x_ptr), C.c_void_p(y_ptr), nvec, precision))

    def heff_apply_part_ptr(self, site, x_ptr: int, y_ptr: int, part: int, nparts: int, nvec: int = 1,
                            precision: int = TNS_FP64):
        """Part `part` of an nparts-way operator-row split of H_eff X (tns_heff_apply_part)."""
        self._check(self._fn("heff_apply_part")(self._h, site, C.c_void_p(x_ptr), C.c_void_p(y_ptr), nvec, precision,
                                                part, nparts))

    def heff_diag_ptr(self, site, d_ptr: int):
        self._check(self._fn("heff_diag")(self._h, site, C.c_void_p(d_ptr)))

    def heff_diag_noalloc_ptr(self, site, d_ptr: int):
        """Allocation-free H_eff diagonal (see tns_heff_diag_noalloc in include/tns.h)."""
        self._check(self._fn("heff_diag_noalloc")(self._h, site, C.c_void_p(d_ptr)))

    def env_arena(self, site, side):
        """(pointer, length) of the left (side 0) or right (side 1) operator arena."""
        p = C.c_void_p()
        n = C.c_longlong()
        self._check(self._fn("env_arena")(self._h, site, side, C.byref(p), C.byref(n)))
        return p.value or 0, n.value

    def heff_adjoint_ptr(self, site, x_ptr, yb_ptr, xb_ptr=0, lb_ptr=0, rb_ptr=0):
        v = lambda p: C.c_void_p(p) if p else None
        self._check(self._fn("heff_adjoint")(self._h, site, v(x_ptr), v(yb_ptr), v(xb_ptr), v(lb_ptr), v(rb_ptr)))

    def sym_eig_ptr(self, sizes, a_ptr: int, z_ptr: int, w_ptr: int):
        """Batched symmetric eigen-decomposition of packed DEVICE matrices (tns_sym_eig)."""
        n = (C.c_int * max(1, len(sizes)))(*sizes)
        self._check(self._fn("sym_eig")(self._h, len(sizes), n, C.c_void_p(a_ptr), C.c_void_p(z_ptr),
                                        C.c_void_p(w_ptr)))

    def rdm_ptr(self, site, psi_ptr: int, N: int, two_body: bool = True):
        """1-RDM (N x N) and, if two_body, the orbit-averaged 2-RDM (N^4) of the
        state given by the MPS and psi (pointer in the library's memory space)
        at step (site, site+1), as dE/dh and 2 dE/dv (tns_rdm)."""
        g = np.zeros(N * N)
        G = np.zeros(N ** 4) if two_body else None
        self._check(self._fn("rdm")(self._h, site, C.c_void_p(psi_ptr), _dptr(g), _dptr(G) if two_body else None))
        return g.reshape(N, N), (G.reshape(N, N, N, N) if two_body else None)

    def heff_flops(self, site):
        f = C.c_double()
        n = C.c_longlong()
        self._check(self._fn("heff_flops")(self._h, site, C.byref(f), C.byref(n)))
        return f.value, n.value

    def davidson_ptr(self, site, x_ptr: int, tol=1e-8, max_iter=200, precision=TNS_FP64):
        e = C.c_double()
        it = C.c_int()
        rc = self._fn("davidson")(self._h, site, C.c_void_p(x_ptr), tol, max_iter, precision, C.byref(e), C.byref(it))
        if rc not in (0, -4):
            self._check(rc)
        return e.value, it.value, rc == 0

    def sweep(self, nsweeps, D, tol=1e-8, max_iter=100, precision=TNS_FP64, cutoff=1e-14, verbose=False, block=1):
        o = SweepOpts(nsweeps, D, tol, max_iter, precision, cutoff, int(verbose), block)
        e = C.c_double()
        st = SweepStats()
        self._check(self._fn("sweep")(self._h, C.byref(o), C.byref(e), C.byref(st)))
        return e.value, st


    def step(self, site, left_to_right, D, tol=1e-8, max_iter=100, precision=TNS_FP64, cutoff=1e-14,
             x0_host_ptr: int = 0, psi_host_ptr: int = 0, block: int = 1):
        """One two-site step; host pointers (0 = none) for the start vector / result."""
        o = SweepOpts(1, D, tol, max_iter, precision, cutoff, 0, block)
        st = StepStats()
        self._check(self._fn("step")(self._h, site, int(left_to_right), C.byref(o),
                                     C.c_void_p(x0_host_ptr) if x0_host_ptr else None,
                                     C.c_void_p(psi_host_ptr) if psi_host_ptr else None, C.byref(st)))
        return st


    def checkpoint_save(self, path: str, site: int = 0, left_to_right: bool = True):
        """Write integrals, MPS and the sweep position to `path` (tns_checkpoint_save)."""
        self._check(self._fn("checkpoint_save")(self._h, os.fsencode(path), site, int(left_to_right)))

    def checkpoint_load(self, path: str):
        """Read a checkpoint into this context; returns (site, left_to_right)."""
        s, d = C.c_int(), C.c_int()
        self._check(self._fn("checkpoint_load")(self._h, os.fsencode(path), C.byref(s), C.byref(d)))
        return s.value, bool(d.value)

    def schedule_stats(self) -> dict:
        """Autotuner counters (tns_schedule_stats)."""
        st = SchedStats()
        self._check(self._fn("schedule_stats")(self._h, C.byref(st)))
        return st.as_dict()

    def set_memory_budget(self, device_bytes: int = 0, host_bytes: int = 0):
        """Device budget and pinned host memory for staged catalogues (0 = none)."""
        self._check(self._fn("set_memory_budget")(self._h, int(device_bytes), int(host_bytes)))

    def memory_stats(self, reset: bool = False) -> dict:
        st = MemStats()
        self._check(self._fn("memory_stats")(self._h, C.byref(st), int(reset)))
        return st.as_dict()

    def psi_guess(self, site, x_host_ptr: int = 0) -> int:
        """Copy the two-site start vector to host memory at x_host_ptr (0: length only)."""
        n = C.c_longlong()
        self._check(self._fn("psi_guess")(self._h, site, C.c_void_p(x_host_ptr) if x_host_ptr else None,
                                          C.byref(n)))
        return n.value


def blocks_to_vector(desc, length, blocks: dict) -> np.ndarray:
    """Pack {(q_l, s1, s2, q_r): array} into the flat layout of psi_layout."""
    x = np.zeros(length)
    for row in desc:
        nl, sl, s1, s2, nr, sr, m, n, off = (int(v) for v in row)
        key = ((nl, sl), s1, s2, (nr, sr))
        if key in blocks:
            x[off:off + m * n] = np.asarray(blocks[key]).ravel()
    return x


def vector_to_blocks(desc, x) -> dict:
    out = {}
    for row in desc:
        nl, sl, s1, s2, nr, sr, m, n, off = (int(v) for v in row)
        out[((nl, sl), s1, s2, (nr, sr))] = np.asarray(x[off:off + m * n]).reshape(m, n)
    return out
