"""The C-ABI library: it loads, exports every symbol include/edac.h declares, and
validates parameters on the host (no GPU call is made by these tests)."""
import ctypes as C
import os
import re

import pytest

from paper_1907_04034_gb300 import binding, cases

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "edac.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(edac_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    binding.build()
    return binding.load()


def test_header_and_binding_agree():
    assert _declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {binding.LIB}").read()
    for name in _declared():
        assert re.search(rf"\bT {name}\b", out), name


def _params(**kw):
    c = cases.channel()
    p = binding.make_params(c.params, binding.EDAC_FP64, c.capacity, 16, True, 0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_workspace_size_for_valid_params(lib):
    n = C.c_size_t(0)
    assert lib.edac_workspace_bytes(C.byref(_params()), C.byref(n)) == 0
    # at least the fp64 master state (~300 B per slot)
    assert n.value > 300 * cases.channel().capacity
    m = C.c_size_t(0)
    assert lib.edac_workspace_bytes(C.byref(_params(precision=binding.EDAC_MIXED)), C.byref(m)) == 0
    assert m.value < n.value


@pytest.mark.parametrize("bad", [dict(dx=0.0), dict(dt=-1.0), dict(x_max=-1.0), dict(precision=7),
                                 dict(capacity=0), dict(eta_reg=0.0), dict(nu=float("nan")),
                                 dict(y_max=0.1)])
def test_invalid_params_are_rejected(lib, bad):
    n = C.c_size_t(0)
    assert lib.edac_workspace_bytes(C.byref(_params(**bad)), C.byref(n)) == 1


def test_create_rejects_missing_or_small_workspace(lib):
    ctx = C.c_void_p()
    p = _params()
    assert lib.edac_create(C.byref(p), None, 0, C.byref(ctx)) == 1
    assert lib.edac_create(C.byref(p), C.c_void_p(4096), 16, C.byref(ctx)) == 1
    assert lib.edac_create(C.byref(p), C.c_void_p(4096 + 8), 1 << 40, C.byref(ctx)) == 1
    assert not ctx.value


def test_null_context_is_an_error(lib):
    assert lib.edac_step(None, 1) == 1


def test_contextless_errors_carry_a_message(lib):
    n = C.c_size_t(0)
    assert lib.edac_workspace_bytes(C.byref(_params(dt=-1.0)), C.byref(n)) == 1
    assert b"must be > 0" in lib.edac_last_error(None)
    assert lib.edac_workspace_bytes(C.byref(_params(periodic_y=1, y_max=0.1)), C.byref(n)) == 1
    assert b"periodic" in lib.edac_last_error(None) or b"empty" in lib.edac_last_error(None)


def test_fma_peak_rejects_bad_arguments_before_any_gpu_call(lib):
    out = C.c_double(-1.0)  # status 1 = EDAC_E_INVALID
    assert lib.edac_fma_peak(7, None, C.byref(out)) == 1
    assert lib.edac_fma_peak(binding.EDAC_PEAK_FP32, None, None) == 1


def test_conversion_check_rejects_null_outputs_before_any_gpu_call(lib):
    out = C.c_uint64(0)  # status 1 = EDAC_E_INVALID
    assert lib.edac_conversion_check(None, 1, 16, None, C.byref(out)) == 1
    assert lib.edac_conversion_check(None, 1, 16, C.byref(out), None) == 1


def test_binding_declares_the_argument_types_of_every_entry(lib):
    # ctypes converts floats and pointers only for declared signatures
    for name in binding.EXPORTS:
        assert getattr(lib, name).argtypes is not None, name


def test_event_log_record_size_and_argument_checks(lib):
    # edac_events_bytes is host-only arithmetic: one record is binding.EVENT_RECORD_BYTES
    nb = C.c_size_t(0)
    assert lib.edac_events_bytes(1, C.byref(nb)) == 0
    assert nb.value == binding.EVENT_RECORD_BYTES
    assert lib.edac_events_bytes(1000, C.byref(nb)) == 0
    assert nb.value == 1000 * binding.EVENT_RECORD_BYTES
    assert lib.edac_events_bytes(-1, C.byref(nb)) == 1
    assert lib.edac_events_bytes(1, None) == 1
    n = C.c_int(0)
    assert lib.edac_read_events(None, 0, None, None, None, None, C.byref(n), None) == 1
    assert lib.edac_events_enable(None, None, 0) == 1


@pytest.fixture
def host_ctx(lib):
    """A context made on the host only: edac_create carves the workspace without touching it, so
    an aligned address that is never dereferenced stands in for device memory."""
    p = _params()
    need = C.c_size_t(0)
    assert lib.edac_workspace_bytes(C.byref(p), C.byref(need)) == 0
    ctx = C.c_void_p()
    assert lib.edac_create(C.byref(p), C.c_void_p(1 << 30), need.value, C.byref(ctx)) == 0
    yield ctx
    lib.edac_destroy(ctx)


EDAC_E_INVALID, EDAC_E_STATE = 1, 6


def test_setters_validate_their_arguments_on_the_host(lib, host_ctx):
    nan = float("nan")
    modes = (C.c_double * 17)(0.01, -0.02)
    ok = lib.edac_set_inlet(host_ctx, 0.0, 3, 2, modes, 0.0, 0.5)
    assert ok == 0
    for args in ((nan, 3, 2, modes, 0.0, 0.5), (0.0, 0, 2, modes, 0.0, 0.5),
                 (0.0, 3, 17, modes, 0.0, 0.5), (0.0, 3, 2, None, 0.0, 0.5),
                 (0.0, 3, 2, modes, 0.0, 0.0), (0.0, 3, -1, modes, 0.0, 0.5)):
        assert lib.edac_set_inlet(host_ctx, *args) == EDAC_E_INVALID, args
    assert b"inlet" in lib.edac_last_error(host_ctx)
    assert lib.edac_set_outlet(host_ctx, 1.0, 5, 0, 6, -1.0) == 0
    for args in ((1.0, 5, 7, 6, -1.0), (1.0, 5, -1, 6, -1.0), (1.0, 0, 0, 6, -1.0),
                 (1.0, 5, 0, 0, -1.0), (1.0, 5, 0, 9, -1.0), (nan, 5, 0, 6, -1.0),
                 (1.0, 5, 0, 6, nan)):
        assert lib.edac_set_outlet(host_ctx, *args) == EDAC_E_INVALID, args
    pulse = (C.c_double * 4)(0.1, 0.2, 0.5, 0.01)
    assert lib.edac_set_inlet_transient(host_ctx, 1, 4, pulse) == 0
    bad_pulse = (C.c_double * 4)(0.1, 0.5, 0.2, 0.01)  # t1 <= t0
    ramp0 = (C.c_double * 1)(0.0)
    for args in ((1, 3, pulse), (1, 4, bad_pulse), (2, 1, ramp0), (2, 1, None), (4, 0, None)):
        assert lib.edac_set_inlet_transient(host_ctx, *args) == EDAC_E_INVALID, args
    assert lib.edac_set_inlet_transient(host_ctx, 0, 0, None) == 0
    assert lib.edac_set_wall(host_ctx, 3, 0, 0.5, 0.0, 2) == 0
    for args in ((0, 0, 0.0, 0.0, 1), (3, 0, 0.0, 0.0, 3), (4, 1, nan, 0.0, 0), (3, 0, 0.0, 0.0, -1)):
        assert lib.edac_set_wall(host_ctx, *args) == EDAC_E_INVALID, args
    assert lib.edac_set_tiling(host_ctx, 8, 128) == 0
    for args in ((0, 128), (17, 128), (8, 100), (8, 32), (8, 288)):
        assert lib.edac_set_tiling(host_ctx, *args) == EDAC_E_INVALID, args


def test_calls_out_of_order_are_state_errors(lib, host_ctx):
    n = C.c_int(-1)
    assert lib.edac_step(host_ctx, 1) == EDAC_E_STATE
    assert b"edac_set_particles" in lib.edac_last_error(host_ctx)
    assert lib.edac_evaluate(host_ctx) == EDAC_E_STATE
    assert lib.edac_get_count(host_ctx, C.byref(n)) == EDAC_E_STATE
    assert lib.edac_step(host_ctx, -1) == EDAC_E_INVALID


def test_derivative_workspaces_are_sized_on_the_host(lib, host_ctx):
    t = C.c_size_t(0)
    assert lib.edac_tangent_workspace_bytes(host_ctx, C.byref(t)) == 0 and t.value > 0
    a = {}
    for nsteps, k in ((400, 50), (800, 50), (400, 25)):
        b = C.c_size_t(0)
        assert lib.edac_adjoint_workspace_bytes(host_ctx, nsteps, k, C.byref(b)) == 0
        a[nsteps, k] = b.value
    assert a[800, 50] > a[400, 50] > 0
    b = C.c_size_t(0)
    assert lib.edac_adjoint_workspace_bytes(host_ctx, 0, 50, C.byref(b)) == EDAC_E_INVALID
    assert lib.edac_adjoint_workspace_bytes(host_ctx, 400, 0, C.byref(b)) == EDAC_E_INVALID


def test_product_fails_loudly_without_its_library(tmp_path):
    """No fallback: with the library missing, loading it (and so making a solver) raises."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1907_04034_gb300 import binding\n"
            "binding.LIB = %r\n"
            "try:\n    binding.load()\nexcept RuntimeError as e:\n    print('raised:', e)\n"
            % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
               str(tmp_path / "libedac.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "raised:" in r.stdout and "build()" in r.stdout


def test_binding_struct_layout_is_the_headers(tmp_path):
    """The ctypes mirror of edac_params has the C header's size and field offsets (compiled
    here with the host C compiler), and make_params fills every field from a case."""
    import subprocess
    fields = [f for f, _ in binding.Params._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'    printf("%s %zu\\n", "{f}", offsetof(edac_params, {f}));' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "edac.h"\n'
                   "int main(void) {\n"
                   '    printf("sizeof %zu\\n", sizeof(edac_params));\n' + body + "\n    return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = os.path.dirname(HEADER)
    r = subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                        text=True).stdout.splitlines())
    assert int(out["sizeof"]) == C.sizeof(binding.Params)
    for f in fields:
        assert int(out[f]) == getattr(binding.Params, f).offset, f
    c = cases.channel()
    p = binding.make_params(c.params, binding.EDAC_MIXED, 1234, 99, True, 0)
    for f in ("x_min", "x_max", "y_min", "y_max", "dx", "hdx", "rho0", "U", "nu", "cs", "alpha",
              "pb", "eta_reg", "gx", "gy", "dt", "periodic_x", "periodic_y", "use_pavg"):
        assert getattr(p, f) == getattr(c.params, f), f
    assert (p.precision, p.capacity, p.max_history, p.use_graphs) == (binding.EDAC_MIXED, 1234, 99, 1)
    assert not p.cuda_stream


def test_binding_constants_are_the_headers(tmp_path):
    """Field ids, kernel ids, statuses, precisions, event kinds, peak kinds and the particle
    tags of the binding and of the cases module are the header's values (compiled here)."""
    import subprocess
    names = (["EDAC_F_" + f.upper() for f in binding.FIELDS] + ["EDAC_NUM_FIELDS"]
             + ["EDAC_K_" + k.upper() for k in binding.KERNELS]
             + list(binding.STATUS.values())
             + ["EDAC_FP64", "EDAC_MIXED", "EDAC_EVENT_DELETE", "EDAC_EVENT_TO_OUTLET",
                "EDAC_EVENT_SPAWN", "EDAC_PEAK_FP32", "EDAC_PEAK_FP64", "EDAC_FLUID",
                "EDAC_INLET", "EDAC_OUTLET", "EDAC_WALL", "EDAC_SLIPWALL",
                "EDAC_OUTLET_HYBRID", "EDAC_OUTLET_DONOTHING", "EDAC_OUTLET_MOD_DONOTHING",
                "EDAC_OUTLET_CHARACTERISTIC", "EDAC_OUTLET_MIRROR", "EDAC_INLET_MODES",
                "EDAC_INLET_PULSE", "EDAC_INLET_RAMP", "EDAC_INLET_VORTEX"])
    src = tmp_path / "consts.c"
    body = "\n".join(f'    printf("%s %d\\n", "{n}", (int)({n}));' for n in names)
    src.write_text('#include <stdio.h>\n#include "edac.h"\nint main(void) {\n' + body +
                   "\n    return 0;\n}\n")
    exe = tmp_path / "consts"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    v = {a: int(b) for a, b in (ln.split() for ln in subprocess.run(
        [str(exe)], capture_output=True, text=True).stdout.splitlines())}
    for i, f in enumerate(binding.FIELDS):
        assert v["EDAC_F_" + f.upper()] == binding.FIELD_ID[f] == i, f
    assert v["EDAC_NUM_FIELDS"] == len(binding.FIELDS)
    for k, i in binding.KERNELS.items():
        assert v["EDAC_K_" + k.upper()] == i, k
    for code, name in binding.STATUS.items():
        assert v[name] == code, name
    assert (v["EDAC_FP64"], v["EDAC_MIXED"]) == (binding.EDAC_FP64, binding.EDAC_MIXED)
    assert (v["EDAC_EVENT_DELETE"], v["EDAC_EVENT_TO_OUTLET"], v["EDAC_EVENT_SPAWN"]) == (
        binding.EVENT_DELETE, binding.EVENT_TO_OUTLET, binding.EVENT_SPAWN)
    assert (v["EDAC_PEAK_FP32"], v["EDAC_PEAK_FP64"]) == (binding.EDAC_PEAK_FP32, binding.EDAC_PEAK_FP64)
    assert [v[n] for n in ("EDAC_FLUID", "EDAC_INLET", "EDAC_OUTLET", "EDAC_WALL",
                           "EDAC_SLIPWALL")] == [cases.FLUID, cases.INLET, cases.OUTLET,
                                                 cases.WALL, cases.SLIPWALL]
    # the outlet kinds of the cases module (Params.outlet_kind) and of the physics driver
    from paper_1907_04034_gb300 import validate
    assert validate.OUTLETS == {"hybrid": v["EDAC_OUTLET_HYBRID"],
                                "donothing": v["EDAC_OUTLET_DONOTHING"],
                                "mod_donothing": v["EDAC_OUTLET_MOD_DONOTHING"],
                                "characteristic": v["EDAC_OUTLET_CHARACTERISTIC"],
                                "mirror": v["EDAC_OUTLET_MIRROR"]}
    assert cases.Params(0.0, 1.0, 0.0, 1.0).outlet_kind == v["EDAC_OUTLET_HYBRID"]
    assert [v[n] for n in ("EDAC_INLET_MODES", "EDAC_INLET_PULSE", "EDAC_INLET_RAMP",
                           "EDAC_INLET_VORTEX")] == [0, 1, 2, 3]
