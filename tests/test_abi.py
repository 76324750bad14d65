"""The C-ABI library builds, loads on a machine without a GPU and exports every
entry point include/*.h declares; host-side argument checks need no device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2010_06697_gb300 import build, rve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(rve_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rve.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"rve_create", "rve_set_material", "rve_solve", "rve_stress", "rve_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(rve.SIGNATURES) >= names


def test_default_options(lib):
    o = rve.rve_default_options()
    assert o.precision == rve.RVE_FP64 and o.rho_policy == rve.RVE_RHO_FIXED
    assert o.max_iter == 1000 and o.rho_kappa == 1.3 and o.rho_tau == 10.0
    assert o.check_every >= 1 and o.use_graph == 1
    # the rest of the header's stated defaults
    assert o.lambda0 == rve.RVE_LAMBDA0_STRESS and o.newton_max == 30 and o.newton_tol == 0.0
    assert o.rho_min == 0.0 and o.mu_ref == 0.0 and o.mixed_switch == 3e-7
    assert o.local_ratio == 0.0 and o.local_fraction == 0.0


def test_workspace_bytes(lib):
    o = rve.rve_default_options()
    b64 = rve.rve_workspace_bytes(3, 128, rve.RVE_NEOHOOKE, o)
    # 2 F + Lambda (9 comps each) + 2 u (3 comps): 33 doubles per voxel at least
    assert b64 >= 33 * 8 * 128 ** 3
    o.precision = rve.RVE_MIXED
    bm = rve.rve_workspace_bytes(3, 128, rve.RVE_NEOHOOKE, o)
    assert bm >= b64 + 33 * 4 * 128 ** 3
    for bad in [(1, 16), (3, 7), (3, 10), (3, 1024), (2, 2)]:
        assert rve.rve_workspace_bytes(bad[0], bad[1], 0, None) == 0


@pytest.mark.parametrize("precision,s", [("fp64", 8), ("mixed", 12), ("fp32", 4)])
def test_workspace_layout_per_voxel(lib, precision, s):
    """The HBM layout: 33 field values per voxel (F twice, Lambda, u~ twice) in each precision
    the handle holds, one phase byte, and under 1 MB of tables, control block and residual
    history at 128^3 (default max_iter); the LCE adds 21 values per voxel (directors twice,
    reference directors, the time step's starting F and n)."""
    V = 128 ** 3
    o = rve.rve_default_options()
    o.precision = rve.PRECISIONS[precision]
    b = rve.rve_workspace_bytes(3, 128, rve.RVE_NEOHOOKE, o)
    assert 33 * s * V + V <= b <= 33 * s * V + V + (1 << 20)
    bl = rve.rve_workspace_bytes(3, 128, rve.RVE_LCE, o)
    assert bl - b == 21 * s * V


@pytest.mark.parametrize("dim,n,model", [(4, 16, 0), (3, 7, 0), (3, 20, 0), (2, 16, 9)])
def test_create_rejects_bad_shapes_without_device(lib, dim, n, model):
    rc, h = rve.rve_create(dim, n, model)
    assert rc == rve.RVE_E_INVALID_ARG and not h.value


def test_create_rejects_bad_options(lib):
    o = rve.rve_default_options()
    o.newton_max = 0
    rc, _ = rve.rve_create(3, 16, 0, o)
    assert rc == rve.RVE_E_INVALID_ARG
    o = rve.rve_default_options()
    o.check_every = 0
    rc, _ = rve.rve_create(3, 16, 0, o)
    assert rc == rve.RVE_E_INVALID_ARG


def test_create_in_rejects_null_and_misaligned_workspaces_without_device(lib):
    """rve_create_in checks the caller's buffer before touching the device: NULL and
    pointers off the 256-byte boundary the field layout assumes are rejected."""
    o = rve.rve_default_options()
    nbytes = rve.rve_workspace_bytes(3, 16, 0, o)
    for ptr in (0, 16, 4096 + 8):
        rc, h = rve.rve_create_in(3, 16, 0, o, None, ptr, nbytes)
        assert rc == rve.RVE_E_INVALID_ARG and not h.value


def test_null_handle_is_rejected(lib):
    assert lib.rve_solve(None, None, ctypes.c_double(1.0), ctypes.c_double(1.0), None) == rve.RVE_E_INVALID_ARG
    assert lib.rve_stress(None, None) == rve.RVE_E_INVALID_ARG
    assert lib.rve_reset(None) == rve.RVE_E_INVALID_ARG
    lib.rve_destroy(None)


def test_strerror(lib):
    for c in range(-8, 1):
        assert len(rve.rve_strerror(c)) > 0


# ------------------------------------------------------------------ binding vs header

_CTYPE = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong,
          "size_t": ctypes.c_size_t, "unsigned": ctypes.c_uint, "float": ctypes.c_float}


def _header_text():
    text = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def _prototypes():
    """name -> list of parameter declarations, from the header's function prototypes."""
    out = {}
    for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rve_\w+)\s*\(([^)]*)\)\s*;", _header_text(), flags=re.M):
        params = [p.strip() for p in m.group(2).replace("\n", " ").split(",") if p.strip()]
        if params == ["void"]:
            params = []
        out[m.group(1)] = params
    return out


def _struct_fields(name):
    m = re.search(r"typedef\s+struct\s+" + name + r"\s*\{(.*?)\}\s*" + name + r"\s*;", _header_text(), flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        mm = re.fullmatch(r"(.+?)\s+(\w+(?:\s*,\s*\w+)*)", decl)  # "double r_p, r_d" declares two
        fields += [(f.strip(), mm.group(1)) for f in mm.group(2).split(",")]
    return fields


def _same_ctype(a, b):
    # ctypes aliases c_longlong to c_long where both are 64-bit: compare size and kind
    floating = (ctypes.c_float, ctypes.c_double)
    return ctypes.sizeof(a) == ctypes.sizeof(b) and (a in floating) == (b in floating)


def test_binding_signatures_match_the_header():
    """Every entry point the binding declares has as many arguments as the header's
    prototype, and scalar arguments have the header's C type (pointers and handles are
    checked by count only)."""
    protos = _prototypes()
    for name, (_, args) in rve.SIGNATURES.items():
        assert name in protos, name
        params = protos[name]
        assert len(args) == len(params), (name, params)
        for a, p in zip(args, params):
            if "*" in p or "[" in p or p.split()[0] in ("rve_t", "rve_batch_t", "rve_server_t"):
                continue
            ctype = " ".join(p.split()[:-1]).replace("const ", "")
            assert ctype in _CTYPE, (name, p)
            assert _same_ctype(a, _CTYPE[ctype]), (name, p, a)


@pytest.mark.parametrize("cname,pyname", [("rve_options", "rve_options"), ("rve_solve_info", "rve_solve_info"),
                                          ("rve_bloch_info", "rve_bloch_info")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors of the header's structs have the same fields, in the same order,
    with the same C types (so the layout the library reads is the one the binding writes)."""
    fields = _struct_fields(cname)
    py = getattr(rve, pyname)._fields_
    assert [f for f, _ in fields] == [f for f, _ in py], cname
    for (f, ctype), (_, pt) in zip(fields, py):
        assert _same_ctype(pt, _CTYPE[ctype]), (cname, f, ctype, pt)


def _header_constants():
    """RVE_* values from the header's #defines and enumerators (explicit values only)."""
    text = _header_text()
    out = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(RVE_\w+)\s+\(?(-?\d+)\)?", text)}
    for body in re.findall(r"enum\s+\w+\s*\{(.*?)\}", text, flags=re.S):
        for m in re.finditer(r"(RVE_\w+)\s*=\s*(-?\d+)", body):
            out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_the_header():
    """Status codes and enumerators the binding names have the header's values."""
    consts = _header_constants()
    assert {"RVE_OK", "RVE_E_INVALID_ARG", "RVE_NEOHOOKE", "RVE_MIXED", "RVE_FIELD_N"} <= set(consts)
    shared = [n for n in consts if hasattr(rve, n)]
    assert len(shared) >= 20
    for n in shared:
        assert getattr(rve, n) == consts[n], n


def test_kernel_class_names_follow_the_header_enum():
    """rve_kernel_times' arrays are indexed by enum rve_kernel_class; the binding labels
    index i with the enumerator's name."""
    consts = _header_constants()
    kc = {n[len("RVE_KCLASS_"):].lower(): v for n, v in consts.items() if n.startswith("RVE_KCLASS_") and n != "RVE_KCLASS_COUNT"}
    assert len(kc) == consts["RVE_KCLASS_COUNT"] == len(rve.KCLASS_NAMES)
    for name, i in kc.items():
        assert rve.KCLASS_NAMES[i] == name, (i, name)


@pytest.mark.parametrize("field,value", [
    ("precision", 3), ("precision", -1), ("rho_policy", 2), ("lambda0", 2), ("max_iter", -1),
    ("newton_max", 1001), ("newton_tol", -1e-3), ("newton_tol", float("nan")), ("rho_kappa", 1.0),
    ("rho_tau", 0.5), ("rho_min", -1.0), ("mu_ref", -1.0), ("mixed_switch", -1.0), ("check_every", 4097),
    ("local_ratio", -0.1), ("local_ratio", float("inf")), ("local_fraction", 1.5), ("local_fraction", float("nan"))])
def test_create_rejects_each_invalid_option_without_device(lib, field, value):
    o = rve.rve_default_options()
    setattr(o, field, value)
    rc, h = rve.rve_create(3, 16, 0, o)
    assert rc == rve.RVE_E_INVALID_ARG and not h.value


@pytest.mark.parametrize("dim,n,model", [(3, 10, 0), (3, 2, 0), (3, 1024, 0), (2, 9, 0), (2, 16, 2), (3, 14, 1)])
def test_create_rejects_grids_and_models_outside_the_contract(lib, dim, n, model):
    """N even of the form 2^a 3^b in [4, 512]; the LCE only in 3D."""
    rc, h = rve.rve_create(dim, n, model)
    assert rc == rve.RVE_E_INVALID_ARG and not h.value


def test_batch_and_server_argument_checks_without_device(lib):
    """Batches need at least one non-NULL handle; servers a non-zero memory budget and
    valid options: checked before any device work."""
    rc, b = rve.rve_batch_create([])
    assert rc == rve.RVE_E_INVALID_ARG and not b.value
    rc, b = rve.rve_batch_create([None, None])
    assert rc == rve.RVE_E_INVALID_ARG and not b.value
    h = ctypes.c_void_p()
    assert lib.rve_server_create(ctypes.byref(h), 0, None, None) == rve.RVE_E_INVALID_ARG and not h.value
    o = rve.rve_default_options()
    o.check_every = 0
    assert lib.rve_server_create(ctypes.byref(h), 1 << 30, ctypes.byref(o), None) == rve.RVE_E_INVALID_ARG
    assert not h.value
    assert lib.rve_batch_solve(None, None, None, ctypes.c_double(1e-8), None) == rve.RVE_E_INVALID_ARG
    lib.rve_batch_destroy(None)
    lib.rve_server_destroy(None)


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without the built library every entry point raises instead of computing
    anything another way."""
    monkeypatch.setattr(rve, "LIB_PATH", os.path.join(ROOT, "does-not-exist", "librve.so"))
    monkeypatch.setattr(rve, "_lib", None)
    with pytest.raises(RuntimeError):
        rve.rve_default_options()
    with pytest.raises(RuntimeError):
        rve.Rve(3, 16, use_torch=False)
