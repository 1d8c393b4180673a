"""CPU oracle for the EDAC / hybrid-outlet step -- TEST INFRASTRUCTURE ONLY.

A plain fp64 C statement of the method (``edac_oracle.c``), loaded with ctypes.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the only common input is the seeded generator module
``paper_1907_04034_gb300.cases``, which carries none of the method's arithmetic.

``OracleSim`` holds one particle system in arrays ordered by ascending particle
id.  Neighbour search is brute force over all pairs by default (the definition);
``neighbor_mode=1`` bins particles into cells of at least 3h and must give the
same lists (pinned by a test), which makes full-size workloads affordable.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "edac_oracle.c")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liboracle.so")
NAVG_MAX = 8
MAX_MODES = 16

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (fp contraction off, OpenMP)."""
    os.makedirs(LIBDIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class CParams(C.Structure):
    _fields_ = [
        ("x_min", C.c_double), ("x_max", C.c_double), ("y_min", C.c_double), ("y_max", C.c_double),
        ("periodic_x", C.c_int), ("periodic_y", C.c_int),
        ("dx", C.c_double), ("hdx", C.c_double), ("rho0", C.c_double), ("U", C.c_double),
        ("nu", C.c_double), ("cs", C.c_double), ("alpha", C.c_double), ("pb", C.c_double),
        ("eta_reg", C.c_double), ("gx", C.c_double), ("gy", C.c_double), ("dt", C.c_double),
        ("use_pavg", C.c_int),
        ("has_inlet", C.c_int), ("x_in", C.c_double), ("n_in_layers", C.c_int),
        ("n_modes", C.c_int), ("modes", C.c_double * MAX_MODES),
        ("inlet_y0", C.c_double), ("inlet_h", C.c_double),
        ("inlet_kind", C.c_int), ("inlet_prm", C.c_double * 4),
        ("has_outlet", C.c_int), ("x_out", C.c_double), ("n_out_layers", C.c_int),
        ("n_avg", C.c_int), ("i_thresh", C.c_double), ("outlet_kind", C.c_int),
        ("moc_u_ref", C.c_double), ("moc_p_ref", C.c_double),
        ("wall_slip", C.c_int * 2), ("wall_u", C.c_double * 2), ("wall_v", C.c_double * 2),
        ("wall_drag", C.c_int * 2), ("drag_length", C.c_double),
        ("neighbor_mode", C.c_int), ("mirror_sign", C.c_int),
    ]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


class CState(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("cap", C.c_int),
        ("x", _DP), ("y", _DP), ("u", _DP), ("v", _DP), ("ut", _DP), ("vt", _DP),
        ("p", _DP), ("m", _DP), ("tag", C.POINTER(C.c_ubyte)), ("id", C.POINTER(C.c_uint64)),
        ("rho", _DP), ("V", _DP), ("nnb", _IP),
        ("au", _DP), ("av", _DP), ("ap", _DP), ("abu", _DP), ("abv", _DP),
        ("fx", _DP), ("fy", _DP),
        ("ring", _DP), ("rpos", _IP),
        ("ubar", _DP), ("vbar", _DP), ("pbar", _DP), ("J2", _DP),
        ("J2p", _DP), ("advp", _DP), ("redp", _IP),
        ("x0", _DP), ("y0", _DP), ("u0", _DP), ("v0", _DP), ("p0", _DP),
        ("next_id", C.c_uint64), ("error", C.c_int), ("t", C.c_double), ("nstep", C.c_int),
        ("ev", C.POINTER(C.c_uint64)), ("ev_cap", C.c_int), ("ev_len", C.c_int),
        ("ev_dropped", C.c_longlong),
    ]


class CHist(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("mass_flux", C.c_double),
                ("n_active", C.c_double), ("n_spawn", C.c_double), ("n_delete", C.c_double),
                ("n_to_outlet", C.c_double), ("pad", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            L.orc_w.restype = C.c_double
            L.orc_w.argtypes = [C.c_double]
            L.orc_dw.restype = C.c_double
            L.orc_dw.argtypes = [C.c_double]
            L.orc_W.restype = C.c_double
            L.orc_W.argtypes = [C.c_double, C.c_double]
            L.orc_dWdr.restype = C.c_double
            L.orc_dWdr.argtypes = [C.c_double, C.c_double]
            for f in ("orc_init", "orc_evaluate"):
                getattr(L, f).argtypes = [C.POINTER(CParams), C.POINTER(CState)]
                getattr(L, f).restype = C.c_int
            L.orc_step.argtypes = [C.POINTER(CParams), C.POINTER(CState), C.c_int, C.POINTER(CHist)]
            L.orc_step.restype = C.c_int
            L.orc_neighbors.argtypes = [C.POINTER(CParams), C.POINTER(CState), _IP, _IP, C.c_int]
            L.orc_neighbors.restype = C.c_int
            L.orc_mirror_points.argtypes = [C.POINTER(CParams), C.POINTER(CState), C.c_int, _DP, _DP,
                                            _DP, _DP, _DP]
            L.orc_mirror_points.restype = C.c_int
            L.orc_outlet_mirror.argtypes = [C.POINTER(CParams), C.POINTER(CState)]
            L.orc_outlet_mirror.restype = C.c_int
            L.orc_probe.argtypes = [C.POINTER(CParams), C.POINTER(CState), C.c_int, _DP, _DP, _DP]
            L.orc_probe.restype = C.c_int
            assert L.orc_sizeof_params() == C.sizeof(CParams), "orc_params layout mismatch"
            assert L.orc_sizeof_state() == C.sizeof(CState), "orc_state layout mismatch"
            assert L.orc_sizeof_hist() == C.sizeof(CHist), "orc_hist layout mismatch"
            _lib = L
    return _lib


def W(r, h):
    return lib().orc_W(float(r), float(h))


def dWdr(r, h):
    return lib().orc_dWdr(float(r), float(h))


def w(q):
    return lib().orc_w(float(q))


def dw(q):
    return lib().orc_dw(float(q))


def make_params(p, neighbor_mode: int = 0, mirror_sign: int = -1) -> CParams:
    """Fill the oracle's parameter struct from a ``cases.Params``."""
    cp = CParams()
    for name in ("x_min", "x_max", "y_min", "y_max", "dx", "hdx", "rho0", "U", "nu", "cs", "alpha",
                 "pb", "eta_reg", "gx", "gy", "dt", "x_in", "x_out", "i_thresh", "drag_length"):
        setattr(cp, name, float(getattr(p, name)))
    for name in ("periodic_x", "periodic_y", "use_pavg", "has_inlet", "n_in_layers", "has_outlet",
                 "n_out_layers", "n_avg", "outlet_kind"):
        setattr(cp, name, int(getattr(p, name)))
    modes = tuple(p.inlet_modes)
    assert len(modes) <= MAX_MODES
    cp.n_modes = len(modes)
    for k, a in enumerate(modes):
        cp.modes[k] = float(a)
    cp.inlet_y0 = float(getattr(p, "inlet_y0", 0.0))
    cp.inlet_h = float(getattr(p, "inlet_h", p.y_max - p.y_min))
    cp.inlet_kind = int(getattr(p, "inlet_kind", 0))
    prm = tuple(getattr(p, "inlet_prm", ()))
    assert len(prm) <= 4
    for k, v in enumerate(prm):
        cp.inlet_prm[k] = float(v)
    ref = tuple(getattr(p, "moc_ref", ())) or (p.U, 0.0)
    cp.moc_u_ref, cp.moc_p_ref = float(ref[0]), float(ref[1])
    for k in range(2):
        cp.wall_slip[k] = int(p.wall_slip[k])
        cp.wall_u[k] = float(p.wall_u[k])
        cp.wall_v[k] = float(p.wall_v[k])
        cp.wall_drag[k] = int(p.wall_drag[k])
    cp.neighbor_mode = int(neighbor_mode)
    cp.mirror_sign = int(mirror_sign)
    return cp


_F64 = ("x", "y", "u", "v", "ut", "vt", "p", "m", "rho", "V", "au", "av", "ap", "abu", "abv",
        "fx", "fy", "ubar", "vbar", "pbar", "J2", "J2p", "advp", "x0", "y0", "u0", "v0", "p0")
_I32 = ("nnb", "rpos", "redp")


class OracleSim:
    """One particle system integrated by the oracle."""

    def __init__(self, case, neighbor_mode: int = 0, params=None, capacity=None,
                 max_events: int = 0):
        self.case = case
        self.params = params if params is not None else case.params
        self.cp = make_params(self.params, neighbor_mode=neighbor_mode)
        cap = int(capacity if capacity is not None else case.capacity)
        n = case.n
        self.a = {k: np.zeros(cap, dtype=np.float64) for k in _F64}
        for k in _I32:
            self.a[k] = np.zeros(cap, dtype=np.int32)
        self.a["tag"] = np.zeros(cap, dtype=np.uint8)
        self.a["id"] = np.zeros(cap, dtype=np.uint64)
        self.a["ring"] = np.zeros(cap * NAVG_MAX * 3, dtype=np.float64)
        for k in ("x", "y", "u", "v", "p", "m", "tag", "id"):
            self.a[k][:n] = getattr(case, k)
        st = CState()
        st.n, st.cap = n, cap
        for k in _F64 + ("ring",):
            setattr(st, k, self.a[k].ctypes.data_as(_DP))
        for k in _I32:
            setattr(st, k, self.a[k].ctypes.data_as(_IP))
        st.tag = self.a["tag"].ctypes.data_as(C.POINTER(C.c_ubyte))
        st.id = self.a["id"].ctypes.data_as(C.POINTER(C.c_uint64))
        st.next_id = 0
        st.error = 0
        # recycling event log (4 words per event: step, kind, id, other id)
        self.a["ev"] = np.zeros(4 * max(int(max_events), 1), dtype=np.uint64)
        st.ev = self.a["ev"].ctypes.data_as(C.POINTER(C.c_uint64)) if max_events > 0 else None
        st.ev_cap = int(max_events)
        st.ev_len = 0
        st.ev_dropped = 0
        self.st = st
        self.history = []
        rc = lib().orc_init(C.byref(self.cp), C.byref(self.st))
        if rc:
            raise RuntimeError(f"oracle init failed ({rc})")

    @property
    def n(self) -> int:
        return int(self.st.n)

    def field(self, name: str) -> np.ndarray:
        return self.a[name][: self.n].copy()

    def fields(self, names=None):
        names = names or ("x", "y", "u", "v", "ut", "vt", "p", "m", "rho", "V", "au", "av",
                          "ap", "abu", "abv", "fx", "fy", "tag", "id", "nnb")
        return {k: self.field(k) for k in names}

    def evaluate(self):
        rc = lib().orc_evaluate(C.byref(self.cp), C.byref(self.st))
        if rc:
            raise RuntimeError(f"oracle evaluate failed ({rc})")

    def step(self, nsteps: int = 1):
        hist = (CHist * max(1, nsteps))()
        rc = lib().orc_step(C.byref(self.cp), C.byref(self.st), int(nsteps), hist)
        recs = [dict(fx=h.fx, fy=h.fy, mass_flux=h.mass_flux, n_active=int(h.n_active),
                     n_spawn=int(h.n_spawn), n_delete=int(h.n_delete),
                     n_to_outlet=int(h.n_to_outlet)) for h in hist[:nsteps]]
        self.history.extend(recs)
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")
        return recs

    def events(self) -> dict:
        """The recycling events logged since the last call, then empties the log: arrays
        step, kind (0 delete, 1 fluid->outlet, 2 spawn), id, other (a spawn's parent id)
        and the number of events dropped for want of room."""
        k = int(self.st.ev_len)
        e = self.a["ev"][: 4 * k].reshape(k, 4).copy()
        out = {"step": e[:, 0].astype(np.int64), "kind": e[:, 1].astype(np.int64),
               "id": e[:, 2].copy(), "other": e[:, 3].copy(), "dropped": int(self.st.ev_dropped)}
        self.st.ev_len = 0
        self.st.ev_dropped = 0
        return out

    def neighbors(self):
        """CSR lists (start[n+1], idx) of array indices, j ascending."""
        n = self.n
        start = np.zeros(n + 1, dtype=np.int32)
        cap = max(1, n) * 128
        idx = np.zeros(cap, dtype=np.int32)
        tot = lib().orc_neighbors(C.byref(self.cp), C.byref(self.st),
                                  start.ctypes.data_as(_IP), idx.ctypes.data_as(_IP), cap)
        if tot > cap:
            idx = np.zeros(tot, dtype=np.int32)
            lib().orc_neighbors(C.byref(self.cp), C.byref(self.st),
                                start.ctypes.data_as(_IP), idx.ctypes.data_as(_IP), tot)
        return start, idx[:tot]

    def mirror_points(self, qx, qy):
        qx = np.ascontiguousarray(qx, dtype=np.float64)
        qy = np.ascontiguousarray(qy, dtype=np.float64)
        pk = np.zeros_like(qx)
        gx = np.zeros_like(qx)
        gy = np.zeros_like(qx)
        lib().orc_mirror_points(C.byref(self.cp), C.byref(self.st), len(qx), qx.ctypes.data_as(_DP),
                                qy.ctypes.data_as(_DP), pk.ctypes.data_as(_DP),
                                gx.ctypes.data_as(_DP), gy.ctypes.data_as(_DP))
        return pk, gx, gy

    def probe(self, qx, qy):
        """Shepard (p, u, v) of the fluid and the fluid count at points: array (n, 4)."""
        qx = np.ascontiguousarray(qx, dtype=np.float64)
        qy = np.ascontiguousarray(qy, dtype=np.float64)
        out = np.zeros((len(qx), 4))
        lib().orc_probe(C.byref(self.cp), C.byref(self.st), len(qx), qx.ctypes.data_as(_DP),
                        qy.ctypes.data_as(_DP), out.ctypes.data_as(_DP))
        return out

    @property
    def t(self) -> float:
        return float(self.st.t)

    def outlet_mirror(self):
        """Run the mirrored outlet update (Sec. 3.2 at the outlet) on the current fields."""
        lib().orc_outlet_mirror(C.byref(self.cp), C.byref(self.st))
