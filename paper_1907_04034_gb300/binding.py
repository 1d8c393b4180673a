"""ctypes binding of the C-ABI library ``libedac.so`` (declared in ``include/edac.h``).

Argument marshalling only: every step of the particle pass runs in the library's
CUDA kernels.  PyTorch provides the device workspace (``torch.empty`` on the CUDA
device, handed to the library as a raw pointer) and the CUDA stream.  There is no
CPU fallback: ``load()`` raises when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, Iterable, Optional

import numpy as np

from . import cases as _cases

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libedac.so")
SOURCES = ("edac_capi.cu", "edac_cells.cu", "edac_pairs.cu", "edac_static.cu", "edac_peaks.cu",
           "edac_tangent.cu", "edac_adjoint.cu", "edac_selfcheck.cu")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

EDAC_FP64, EDAC_MIXED = 0, 1
STATUS = {0: "EDAC_OK", 1: "EDAC_E_INVALID", 2: "EDAC_E_CAPACITY", 3: "EDAC_E_CUDA",
          4: "EDAC_E_NONFINITE", 5: "EDAC_E_TIMEOUT", 6: "EDAC_E_STATE", 7: "EDAC_E_DOMAIN"}
FIELDS = ("x", "y", "u", "v", "ut", "vt", "p", "m", "rho", "vol", "au", "av", "ap", "abu", "abv",
          "fx", "fy", "nnb", "ubar", "vbar", "pbar", "J2", "J2p", "advp", "redp", "rpos")
FIELD_ID = {k: i for i, k in enumerate(FIELDS)}
KERNELS = {"pass_a": 0, "pass_b": 1, "rebuild": 2, "boundary": 3, "stage": 4, "recycle": 5}
EVENT_DELETE, EVENT_TO_OUTLET, EVENT_SPAWN = 0, 1, 2
EVENT_RECORD_BYTES = 24

# every symbol the header declares
EXPORTS = ("edac_workspace_bytes", "edac_create", "edac_set_inlet", "edac_set_outlet",
           "edac_set_wall", "edac_set_particles", "edac_step", "edac_evaluate", "edac_get_count",
           "edac_read_state", "edac_read_history", "edac_neighbor_scratch_bytes",
           "edac_read_neighbors", "edac_profile", "edac_read_profile", "edac_launch_count",
           "edac_density_static", "edac_fma_peak", "edac_conversion_check", "edac_set_tiling",
           "edac_autotune",
           "edac_batch_create", "edac_batch_step", "edac_batch_launch_count", "edac_batch_destroy",
           "edac_batch_workspace_bytes", "edac_batch_create_fused",
           "edac_set_inlet_transient", "edac_set_outlet_reference", "edac_probe",
           "edac_tangent_workspace_bytes", "edac_tangent_enable", "edac_step_tangent",
           "edac_read_tangent_history", "edac_adjoint_workspace_bytes", "edac_adjoint_run",
           "edac_events_bytes", "edac_events_enable", "edac_read_events",
           "edac_last_error", "edac_destroy")


class EdacError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libedac.so for sm_103a (the translation units in parallel)."""
    os.makedirs(LIBDIR, exist_ok=True)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [
        os.path.join(CSRC, "edac_internal.cuh"), os.path.join(INCLUDE, "edac.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in deps):
            return LIB
    nvcc = _nvcc()
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-pthread",
             "-I" + INCLUDE, "-I" + CSRC]
    objs = []

    def comp(src):
        obj = os.path.join(LIBDIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(comp, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [
        ("x_min", C.c_double), ("x_max", C.c_double), ("y_min", C.c_double), ("y_max", C.c_double),
        ("periodic_x", C.c_int), ("periodic_y", C.c_int),
        ("dx", C.c_double), ("hdx", C.c_double), ("rho0", C.c_double), ("U", C.c_double),
        ("nu", C.c_double), ("cs", C.c_double), ("alpha", C.c_double), ("pb", C.c_double),
        ("eta_reg", C.c_double), ("gx", C.c_double), ("gy", C.c_double), ("dt", C.c_double),
        ("use_pavg", C.c_int), ("precision", C.c_int), ("capacity", C.c_int),
        ("max_history", C.c_int), ("use_graphs", C.c_int), ("cuda_stream", C.c_void_p),
    ]


_lock = threading.Lock()
_lib = None

_P = C.c_void_p
_DP = C.POINTER(C.c_double)


def load(path: Optional[str] = None):
    """Load libedac.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libedac.so not found at {p}: run build() (nvcc, sm_103a) first")
        L = C.CDLL(p)
        i32, i64, sz = C.c_int, C.c_int64, C.c_size_t
        L.edac_workspace_bytes.argtypes = [C.POINTER(Params), C.POINTER(sz)]
        L.edac_create.argtypes = [C.POINTER(Params), _P, sz, C.POINTER(_P)]
        L.edac_set_inlet.argtypes = [_P, C.c_double, i32, i32, _DP, C.c_double, C.c_double]
        L.edac_set_outlet.argtypes = [_P, C.c_double, i32, i32, i32, C.c_double]
        L.edac_set_wall.argtypes = [_P, i32, i32, C.c_double, C.c_double, i32]
        L.edac_set_particles.argtypes = [_P, i32] + [_DP] * 6 + [C.POINTER(C.c_uint8),
                                                                 C.POINTER(C.c_uint64)]
        L.edac_step.argtypes = [_P, i32]
        L.edac_evaluate.argtypes = [_P]
        L.edac_get_count.argtypes = [_P, C.POINTER(i32)]
        L.edac_read_state.argtypes = [_P, i32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint8), i32,
                                      C.POINTER(i32), C.POINTER(_DP), C.POINTER(i32)]
        L.edac_read_history.argtypes = [_P, i32, _DP, _DP, _DP] + [C.POINTER(i32)] * 5
        L.edac_neighbor_scratch_bytes.argtypes = [_P, C.POINTER(sz)]
        L.edac_read_neighbors.argtypes = [_P, _P, sz, i32, C.POINTER(i64), i64,
                                          C.POINTER(C.c_uint64), C.POINTER(i32), C.POINTER(i64)]
        L.edac_profile.argtypes = [_P, i32, i32]
        L.edac_read_profile.argtypes = [_P, i32, _DP, C.POINTER(i64), i32]
        L.edac_launch_count.argtypes = [_P, C.POINTER(i64)]
        L.edac_density_static.argtypes = [C.POINTER(Params), i32] + [_P] * 6
        L.edac_fma_peak.argtypes = [i32, _P, _DP]
        L.edac_conversion_check.argtypes = [_P, i32, C.c_uint64, C.POINTER(C.c_uint64),
                                            C.POINTER(C.c_uint64)]
        L.edac_set_tiling.argtypes = [_P, i32, i32]
        L.edac_autotune.argtypes = [_P, i32, C.POINTER(i32), C.POINTER(i32), _DP]
        L.edac_batch_create.argtypes = [C.POINTER(_P), i32, _P, C.POINTER(_P)]
        L.edac_batch_workspace_bytes.argtypes = [i32, C.POINTER(sz)]
        L.edac_batch_create_fused.argtypes = [C.POINTER(_P), i32, _P, _P, sz, C.POINTER(_P)]
        L.edac_batch_step.argtypes = [_P, i32]
        L.edac_batch_launch_count.argtypes = [_P, C.POINTER(i64)]
        L.edac_batch_destroy.argtypes = [_P]
        L.edac_set_inlet_transient.argtypes = [_P, i32, i32, _DP]
        L.edac_set_outlet_reference.argtypes = [_P, C.c_double, C.c_double]
        L.edac_probe.argtypes = [_P, i32, _DP, _DP, _DP]
        L.edac_tangent_workspace_bytes.argtypes = [_P, C.POINTER(sz)]
        L.edac_tangent_enable.argtypes = [_P, _P, sz]
        L.edac_step_tangent.argtypes = [_P, i32]
        L.edac_read_tangent_history.argtypes = [_P, i32, _DP, _DP, C.POINTER(i32)]
        L.edac_adjoint_workspace_bytes.argtypes = [_P, i32, i32, C.POINTER(sz)]
        L.edac_adjoint_run.argtypes = [_P, _P, sz, i32, i32, _DP, _DP, _DP, C.c_double, C.c_double,
                                       _DP, _DP]
        L.edac_events_bytes.argtypes = [i32, C.POINTER(sz)]
        L.edac_events_enable.argtypes = [_P, _P, sz]
        L.edac_read_events.argtypes = [_P, i32, C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                       C.POINTER(i32), C.POINTER(i64)]
        L.edac_last_error.argtypes = [_P]
        L.edac_last_error.restype = C.c_char_p
        L.edac_destroy.argtypes = [_P]
        L.edac_destroy.restype = None
        L.edac_batch_destroy.restype = None
        for name in EXPORTS:
            if name not in ("edac_last_error", "edac_destroy", "edac_batch_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def make_params(p: "_cases.Params", precision: int, capacity: int, max_history: int,
                use_graphs: bool, stream_ptr: int) -> Params:
    q = Params()
    for name in ("x_min", "x_max", "y_min", "y_max", "dx", "hdx", "rho0", "U", "nu", "cs", "alpha",
                 "pb", "eta_reg", "gx", "gy", "dt"):
        setattr(q, name, float(getattr(p, name)))
    q.periodic_x = int(p.periodic_x)
    q.periodic_y = int(p.periodic_y)
    q.use_pavg = int(p.use_pavg)
    q.precision = int(precision)
    q.capacity = int(capacity)
    q.max_history = int(max_history)
    q.use_graphs = int(bool(use_graphs))
    q.cuda_stream = stream_ptr or None
    return q


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def density_static(case, device: str = "cuda:0", stream=None):
    """Summation density, volume and neighbour count through edac_density_static.

    The call itself allocates nothing on the device: its scratch is the library's static
    array.  This helper (the caller) owns the input and output tensors.  Returns numpy
    arrays (rho, vol, nnb) in the order of the case's particles.
    """
    import torch

    lib = load()
    dev = torch.device(device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    p = make_params(case.params, EDAC_FP64, max(1, case.n), 1, False, st.cuda_stream)
    x = torch.as_tensor(np.ascontiguousarray(case.x, dtype=np.float64), device=dev)
    y = torch.as_tensor(np.ascontiguousarray(case.y, dtype=np.float64), device=dev)
    m = torch.as_tensor(np.ascontiguousarray(case.m, dtype=np.float64), device=dev)
    rho = torch.empty_like(x)
    vol = torch.empty_like(x)
    nnb = torch.empty(case.n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.device(dev):
        rc = lib.edac_density_static(C.byref(p), int(case.n), C.c_void_p(x.data_ptr()),
                                     C.c_void_p(y.data_ptr()), C.c_void_p(m.data_ptr()),
                                     C.c_void_p(rho.data_ptr()), C.c_void_p(vol.data_ptr()),
                                     C.c_void_p(nnb.data_ptr()))
    if rc != 0:
        raise EdacError(rc, "edac_density_static")
    return rho.cpu().numpy(), vol.cpu().numpy(), nnb.cpu().numpy()


EDAC_PEAK_FP32, EDAC_PEAK_FP64 = 0, 1


def fma_peak(kind: int, device: str = "cuda:0", stream=None) -> float:
    """Measured FMA-pipe peak of the device in TFLOP/s (edac_fma_peak): kind EDAC_PEAK_FP32
    or EDAC_PEAK_FP64.  About 0.1 s of GPU time; synchronises the stream."""
    import torch

    lib = load()
    dev = torch.device(device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    out = C.c_double(0.0)
    with torch.cuda.device(dev):
        rc = lib.edac_fma_peak(int(kind), C.c_void_p(st.cuda_stream), C.byref(out))
    if rc != 0:
        raise EdacError(rc, "edac_fma_peak")
    return float(out.value)


def conversion_check(all_floats: bool = True, n_doubles: int = 1 << 28,
                     device: str = "cuda:0") -> tuple:
    """(float, double) mismatch counts of the library's integer-pipe conversions against the
    hardware ones (edac_conversion_check)."""
    import torch

    lib = load()
    dev = torch.device(device)
    st = torch.cuda.current_stream(dev)
    a, b = C.c_uint64(0), C.c_uint64(0)
    with torch.cuda.device(dev):
        rc = lib.edac_conversion_check(C.c_void_p(st.cuda_stream), int(bool(all_floats)),
                                       int(n_doubles), C.byref(a), C.byref(b))
    if rc != 0:
        raise EdacError(rc, "edac_conversion_check")
    return int(a.value), int(b.value)


class Solver:
    """One particle system on one GPU, driven through the C ABI."""

    def __init__(self, case, precision: str = "fp64", use_graphs: bool = True,
                 max_history: int = 4096, capacity: Optional[int] = None, device: str = "cuda:0",
                 stream=None, params=None):
        import torch  # device memory and streams only

        self.lib = load()
        self.torch = torch
        self.case = case
        self.params = params if params is not None else case.params
        self.event_log = None
        self.precision = {"fp64": EDAC_FP64, "mixed": EDAC_MIXED}[precision]
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        cap = int(capacity if capacity is not None else case.capacity)
        self.cparams = make_params(self.params, self.precision, cap, max_history, use_graphs,
                                   self.stream.cuda_stream)
        nbytes = C.c_size_t(0)
        self._check(self.lib.edac_workspace_bytes(C.byref(self.cparams), C.byref(nbytes)), None)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            self._check(self.lib.edac_create(C.byref(self.cparams), C.c_void_p(self.workspace.data_ptr()),
                                             nbytes.value, C.byref(self.ctx)), None)
        p = self.params
        if p.has_inlet:
            modes = np.ascontiguousarray(p.inlet_modes, dtype=np.float64)
            self._call("edac_set_inlet", p.x_in, p.n_in_layers, len(modes),
                       _ptr(modes, C.c_double) if len(modes) else None, p.inlet_y0, p.inlet_h)
        if p.has_inlet and int(getattr(p, "inlet_kind", 0)) != 0:
            prm = np.ascontiguousarray(p.inlet_prm, dtype=np.float64)
            self._call("edac_set_inlet_transient", int(p.inlet_kind), len(prm),
                       _ptr(prm, C.c_double) if len(prm) else None)
        if p.has_outlet:
            self._call("edac_set_outlet", p.x_out, p.n_out_layers, int(p.outlet_kind), p.n_avg,
                       p.i_thresh)
            ref = tuple(getattr(p, "moc_ref", ())) or (p.U, 0.0)
            self._call("edac_set_outlet_reference", float(ref[0]), float(ref[1]))
        for tagv, w in ((_cases.WALL, 0), (_cases.SLIPWALL, 1)):
            self._call("edac_set_wall", tagv, int(p.wall_slip[w]), float(p.wall_u[w]),
                       float(p.wall_v[w]), int(p.wall_drag[w]))
        self.upload(case)

    # -------------------------------------------------------------------------- plumbing
    def _check(self, rc, ctx):
        if rc != 0:
            msg = self.lib.edac_last_error(ctx).decode()
            raise EdacError(rc, msg)

    def _call(self, name, *args):
        with self.torch.cuda.device(self.device):
            rc = getattr(self.lib, name)(self.ctx, *args)
        self._check(rc, self.ctx)
        return rc

    # ------------------------------------------------------------------------------- API
    def upload(self, case):
        a = {k: np.ascontiguousarray(getattr(case, k)) for k in ("x", "y", "u", "v", "p", "m")}
        tag = np.ascontiguousarray(case.tag, dtype=np.uint8)
        ids = np.ascontiguousarray(case.id, dtype=np.uint64)
        self._call("edac_set_particles", int(case.n), *[_ptr(a[k].astype(np.float64), C.c_double)
                                                        if a[k].dtype != np.float64 else _ptr(a[k], C.c_double)
                                                        for k in ("x", "y", "u", "v", "p", "m")],
                   _ptr(tag, C.c_uint8), _ptr(ids, C.c_uint64))

    def step(self, n: int = 1):
        self._call("edac_step", int(n))

    def evaluate(self):
        self._call("edac_evaluate")

    def count(self) -> int:
        n = C.c_int(0)
        self._call("edac_get_count", C.byref(n))
        return n.value

    def state(self, fields: Iterable[str] = ("x", "y", "u", "v", "p")) -> Dict[str, np.ndarray]:
        """Live particles in ascending id order: id, tag and the requested fields."""
        fields = list(fields)
        cap = int(self.cparams.capacity)
        ids = np.empty(cap, dtype=np.uint64)
        tags = np.empty(cap, dtype=np.uint8)
        outs = [np.empty(cap, dtype=np.float64) for _ in fields]
        fid = (C.c_int * max(1, len(fields)))(*[FIELD_ID[f] for f in fields])
        optr = (_DP * max(1, len(fields)))(*[_ptr(o, C.c_double) for o in outs])
        n = C.c_int(0)
        self._call("edac_read_state", cap, _ptr(ids, C.c_uint64), _ptr(tags, C.c_uint8),
                   len(fields), fid, optr, C.byref(n))
        k = n.value
        out = {"id": ids[:k], "tag": tags[:k]}
        for f, o in zip(fields, outs):
            out[f] = o[:k]
        return out

    def history(self, max_steps: Optional[int] = None):
        m = int(max_steps or self.cparams.max_history)
        fx, fy, mf = (np.zeros(m) for _ in range(3))
        na, sp, dl, to = (np.zeros(m, dtype=np.int32) for _ in range(4))
        ns = C.c_int(0)
        self._call("edac_read_history", m, _ptr(fx, C.c_double), _ptr(fy, C.c_double),
                   _ptr(mf, C.c_double), _ptr(na, C.c_int), _ptr(sp, C.c_int), _ptr(dl, C.c_int),
                   _ptr(to, C.c_int), C.byref(ns))
        k = ns.value
        return dict(fx=fx[:k], fy=fy[:k], mass_flux=mf[:k], n_active=na[:k], n_spawn=sp[:k],
                    n_delete=dl[:k], n_to_outlet=to[:k])

    def neighbors(self):
        """(ids ascending, CSR start, neighbour ids) built with the pair kernels' test."""
        nb = C.c_size_t(0)
        self._call("edac_neighbor_scratch_bytes", C.byref(nb))
        scratch = self.torch.empty(int(nb.value), dtype=self.torch.uint8, device=self.device)
        cap_n = int(self.cparams.capacity)
        start = np.zeros(cap_n + 1, dtype=np.int64)
        cap_ids = max(1, (int(nb.value) - 8 * (cap_n + 1)) // 8 + cap_n + 64)
        ids = np.zeros(cap_ids, dtype=np.uint64)
        n = C.c_int(0)
        tot = C.c_int64(0)
        self._call("edac_read_neighbors", C.c_void_p(scratch.data_ptr()), nb.value, cap_n,
                   _ptr(start, C.c_int64), cap_ids, _ptr(ids, C.c_uint64), C.byref(n), C.byref(tot))
        del scratch
        return start[: n.value + 1].copy(), ids[: tot.value].copy()

    def profile(self, kernel: str, enable: bool = True):
        self._call("edac_profile", KERNELS[kernel], int(enable))

    def read_profile(self, kernel: str, reset: bool = True):
        ms = C.c_double(0)
        ln = C.c_int64(0)
        self._call("edac_read_profile", KERNELS[kernel], C.byref(ms), C.byref(ln), int(reset))
        return ms.value, ln.value

    def probe(self, xs, ys) -> np.ndarray:
        """Shepard (p, u, v) of the fluid and the fluid count at points (edac_probe):
        array (n, 4)."""
        xs = np.ascontiguousarray(xs, dtype=np.float64)
        ys = np.ascontiguousarray(ys, dtype=np.float64)
        out = np.zeros((len(xs), 4))
        self._call("edac_probe", len(xs), _ptr(xs, C.c_double), _ptr(ys, C.c_double),
                   _ptr(out, C.c_double))
        return out

    # ------------------------------------------------------------------ event log
    def events_enable(self, max_events: int):
        """Log the recycling events of every step (edac_events_enable) into a device tensor
        of max_events records; 0 switches the log off."""
        if max_events <= 0:
            self._call("edac_events_enable", None, 0)
            self.event_log = None
            return
        nb = C.c_size_t(0)
        self._check(self.lib.edac_events_bytes(int(max_events), C.byref(nb)), None)
        with self.torch.cuda.device(self.device):
            log = self.torch.empty(int(nb.value), dtype=self.torch.uint8, device=self.device)
        self._call("edac_events_enable", C.c_void_p(log.data_ptr()), nb.value)
        self.event_log = log

    def events(self) -> dict:
        """The logged events since the last call, oldest first (edac_read_events): arrays
        step, kind (EVENT_*), id, other, and the number of events dropped."""
        cap = int(self.event_log.numel()) // EVENT_RECORD_BYTES if self.event_log is not None else 0
        step = np.zeros(max(cap, 1), np.int32)
        kind = np.zeros(max(cap, 1), np.int32)
        ids = np.zeros(max(cap, 1), np.uint64)
        other = np.zeros(max(cap, 1), np.uint64)
        n = C.c_int(0)
        dropped = C.c_int64(0)
        self._call("edac_read_events", cap, _ptr(step, C.c_int), _ptr(kind, C.c_int),
                   _ptr(ids, C.c_uint64), _ptr(other, C.c_uint64), C.byref(n), C.byref(dropped))
        k = n.value
        return {"step": step[:k].copy(), "kind": kind[:k].copy(), "id": ids[:k].copy(),
                "other": other[:k].copy(), "dropped": int(dropped.value)}

    # ------------------------------------------------------------ tangent-linear model
    def tangent_enable(self):
        """Allocate the tangent workspace and set the tangents (edac_tangent_enable)."""
        nb = C.c_size_t(0)
        self._call("edac_tangent_workspace_bytes", C.byref(nb))
        with self.torch.cuda.device(self.device):
            self.tangent_ws = self.torch.empty(int(nb.value), dtype=self.torch.uint8,
                                               device=self.device)
        self._call("edac_tangent_enable", C.c_void_p(self.tangent_ws.data_ptr()), nb.value)

    def step_tangent(self, n: int = 1):
        self._call("edac_step_tangent", int(n))

    def tangent_history(self, max_steps: Optional[int] = None):
        """(dFx/da, dFy/da): arrays (steps, 8) aligned with history()."""
        m = int(max_steps or self.cparams.max_history)
        dfx = np.zeros((m, 8))
        dfy = np.zeros((m, 8))
        ns = C.c_int(0)
        self._call("edac_read_tangent_history", m, _ptr(dfx, C.c_double), _ptr(dfy, C.c_double),
                   C.byref(ns))
        return dfx[: ns.value].copy(), dfy[: ns.value].copy()

    def adjoint(self, nsteps: int, checkpoint_every: int = 50, w_fx=None, w_fy=None, w_pe=None,
                pe_window=(0.0, 0.0)):
        """Reverse-mode gradient (edac_adjoint_run) of L = sum_n w_fx[n] F_x^n + w_fy[n] F_y^n
        + w_pe[n] sum_{fluid in pe_window} p^2 over nsteps steps from the freshly uploaded
        state, with respect to the 8 inlet modes: (L, dL/da).  The workspace (checkpoints
        every checkpoint_every steps) is a torch tensor freed on return."""
        torch = self.torch
        nb = C.c_size_t(0)
        self._call("edac_adjoint_workspace_bytes", int(nsteps), int(checkpoint_every), C.byref(nb))
        with torch.cuda.device(self.device):
            ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)

        def arr(w):
            if w is None:
                return None
            a = np.ascontiguousarray(w, dtype=np.float64)
            assert a.shape == (int(nsteps),)
            return a

        wx, wy, wp = arr(w_fx), arr(w_fy), arr(w_pe)
        loss = C.c_double(0.0)
        grad = np.zeros(8)
        self._call("edac_adjoint_run", C.c_void_p(ws.data_ptr()), nb.value, int(nsteps),
                   int(checkpoint_every), *[_ptr(a, C.c_double) if a is not None else None
                                            for a in (wx, wy, wp)],
                   float(pe_window[0]), float(pe_window[1]), C.byref(loss), _ptr(grad, C.c_double))
        del ws
        return loss.value, grad

    def set_tiling(self, tile_cells: int, threads: int):
        """Tiling of the mixed pair passes (edac_set_tiling)."""
        self._call("edac_set_tiling", int(tile_cells), int(threads))

    def autotune(self, trials: int = 3):
        """Pick the fastest tiling by timing evaluations (edac_autotune); returns
        (tile_cells, threads, ms per evaluation)."""
        tx, tpb, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
        self._call("edac_autotune", int(trials), C.byref(tx), C.byref(tpb), C.byref(ms))
        return tx.value, tpb.value, ms.value

    def launch_count(self) -> int:
        c = C.c_int64(0)
        self._call("edac_launch_count", C.byref(c))
        return c.value

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            with self.torch.cuda.device(self.device):
                self.lib.edac_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent systems advanced together, one graph launch per step (edac_batch_step).
    fused=False: the graph's branches are the members' steps (edac_batch_create); fused=True:
    each kernel of the step is launched once over all members (edac_batch_create_fused, whose
    member tables live in a torch-allocated device workspace).  The members are ``Solver``
    objects on one device, each with its own stream; configure them first."""

    def __init__(self, solvers, stream=None, fused: bool = False):
        import torch

        self.lib = load()
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        self.device = dev
        # torch hands out streams from per-priority pools: the members' default-priority
        # streams may repeat (that only serialises them), the batch's own comes from the
        # high-priority pool so that it differs from every member's
        self.stream = stream if stream is not None else torch.cuda.Stream(dev, priority=-1)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        self.b = C.c_void_p()
        self.fused = bool(fused)
        self.workspace = None
        with torch.cuda.device(dev):
            if self.fused:
                nb = C.c_size_t(0)
                rc = self.lib.edac_batch_workspace_bytes(len(self.solvers), C.byref(nb))
                if rc != 0:
                    raise EdacError(rc, self.lib.edac_last_error(None).decode())
                self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=dev)
                rc = self.lib.edac_batch_create_fused(
                    arr, len(self.solvers), C.c_void_p(self.stream.cuda_stream),
                    C.c_void_p(self.workspace.data_ptr()), nb.value, C.byref(self.b))
            else:
                rc = self.lib.edac_batch_create(arr, len(self.solvers),
                                                C.c_void_p(self.stream.cuda_stream), C.byref(self.b))
        if rc != 0:
            raise EdacError(rc, self.lib.edac_last_error(None).decode())

    def step(self, n: int = 1):
        import torch

        with torch.cuda.device(self.device):
            rc = self.lib.edac_batch_step(self.b, int(n))
        if rc != 0:
            raise EdacError(rc, self.lib.edac_last_error(None).decode())

    def kernels_per_step(self) -> int:
        k = C.c_int64(0)
        rc = self.lib.edac_batch_launch_count(self.b, C.byref(k))
        if rc != 0:
            raise EdacError(rc, "edac_batch_launch_count")
        return k.value

    def close(self):
        if getattr(self, "b", None) and self.b.value:
            import torch

            with torch.cuda.device(self.device):
                self.lib.edac_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
