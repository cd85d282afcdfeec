"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/adsgb.h declares, and its pure-host helpers behave."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adsgb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("typedef")))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    return _lib.load()


def test_header_parses():
    names = declared_functions()
    for must in ("ads_init", "ads_saturation_step", "crvpinn_pretrain", "crvpinn_pressure_update",
                 "hybrid_step", "ads_destroy", "ads_get"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2604_20731_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in adsgb.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_status_strings(lib):
    assert lib.ads_status_str(0) == b"ok"
    assert lib.ads_status_str(5) == b"timeout"
    assert lib.ads_status_str(8) == b"checkpoint file error"
    assert lib.ads_status_str(99) == b"unknown"


def test_struct_layouts_match_header():
    from paper_2604_20731_gb300 import _lib
    # ads_source: 3 doubles + sigma + rate + int (padded to 8)
    assert C.sizeof(_lib.ads_source) == 48
    assert C.sizeof(_lib.crvpinn_params) == 16  # width, hidden_layers, dtype, act_chunks
    assert C.sizeof(_lib.hybrid_stats) == 32


def test_hbm_estimate_and_validation(lib):
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import make_params
    sc = scn.make_scenario(2, 256)
    p = make_params(sc, "f64")
    crv = _lib.crvpinn_params(64, 4, _lib.ADS_F32)
    b = lib.ads_hbm_estimate(C.byref(p), C.byref(crv))
    assert 10e6 < b < 2e9
    b0 = lib.ads_hbm_estimate(C.byref(p), None)
    assert 0 < b0 < b
    # activation recomputation: the stored activations shrink to one chunk
    all_acts = _lib.crvpinn_params(128, 4, _lib.ADS_BF16, 1)
    chunked = _lib.crvpinn_params(128, 4, _lib.ADS_BF16, 4)
    assert lib.ads_hbm_estimate(C.byref(p), C.byref(chunked)) < lib.ads_hbm_estimate(C.byref(p), C.byref(all_acts))
    assert lib.ads_hbm_estimate(C.byref(p), C.byref(_lib.crvpinn_params(128, 4, _lib.ADS_BF16, -1))) == 0
    p.n = 1  # invalid
    assert lib.ads_hbm_estimate(C.byref(p), C.byref(crv)) == 0
    p.n = 256
    crv.width = 96  # unsupported width
    assert lib.ads_hbm_estimate(C.byref(p), C.byref(crv)) == 0


def test_init_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import make_params
    sc = scn.make_scenario(2, 8)
    p = make_params(sc)
    out = C.c_void_p()
    assert lib.ads_init(C.byref(p), None, None, None, None, None, C.byref(out)) == 1  # K missing
    p.dim = 4
    K = (C.c_double * 81)(*([1.0] * 81))
    assert lib.ads_init(C.byref(p), None, K, None, None, None, C.byref(out)) == 7
    p.dim = 2
    p.mu_g = -1.0
    assert lib.ads_init(C.byref(p), None, K, None, None, None, C.byref(out)) == 1
    p.mu_g = 1.0
    K[3] = float("nan")
    assert lib.ads_init(C.byref(p), None, K, None, None, None, C.byref(out)) == 4
    assert not out.value


C_CONSUMER = r"""
#include <stdio.h>
#include <string.h>
#include "adsgb.h"

int main(void) {
  ads_params p;
  crvpinn_params c = {64, 4, ADS_F32, 0};
  ads_ctx* ctx = NULL;
  ads_status st;
  size_t b, b0;
  memset(&p, 0, sizeof p);
  p.dim = 2;
  p.n = 256;
  p.phi = 0.2;
  p.mu_w = 6.4;
  p.mu_g = 1.0;
  p.rho_w = 1.0;
  p.rho_g = 0.46;
  p.grav_sign = 1.0;
  p.kz_ratio = 1.0;
  p.n_src = 1;
  p.src[0].center[0] = 0.25;
  p.src[0].center[1] = 0.25;
  p.src[0].sigma = 0.03;
  p.src[0].rate = 1.0;
  p.src[0].kind = 0;
  p.ads_dtype = ADS_F64;
  b = ads_hbm_estimate(&p, &c);
  b0 = ads_hbm_estimate(&p, NULL);
  /* a missing K is refused before any CUDA call */
  st = ads_init(&p, NULL, NULL, NULL, NULL, NULL, &ctx);
  printf("%s %lu %lu %lu %lu %lu %lu %lu %d %d\n", ads_status_str(ADS_OK), (unsigned long)b,
         (unsigned long)b0, (unsigned long)sizeof(ads_params), (unsigned long)sizeof(crvpinn_params),
         (unsigned long)sizeof(hybrid_params), (unsigned long)sizeof(hybrid_stats),
         (unsigned long)sizeof(ads_allocator), (int)st, ctx == NULL);
  return 0;
}
"""


def test_c99_consumer_compiles_links_and_runs(lib, tmp_path):
    """The header is plain C99 and the library links into a C program; its
    struct sizes agree with the binding's and the host-only calls work."""
    import shutil
    import subprocess
    from paper_2604_20731_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    pkg = os.path.dirname(_lib.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-L", pkg, "-ladsgb",
                    f"-Wl,-rpath,{pkg}", "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == "ok"
    b, b0 = int(out[1]), int(out[2])
    assert 0 < b0 < b
    assert [int(v) for v in out[3:8]] == [C.sizeof(_lib.ads_params), C.sizeof(_lib.crvpinn_params),
                                          C.sizeof(_lib.hybrid_params), C.sizeof(_lib.hybrid_stats),
                                          C.sizeof(_lib.ads_allocator)]
    assert int(out[8]) == 1 and int(out[9]) == 1  # ADS_ERR_INVALID_ARG, no context


def _prototypes():
    """name -> parameter count for every function prototype in the header."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src)  # typedefs (incl. function-pointer types)
    out = {}
    for m in re.finditer(r"([a-z_][a-z0-9_]*)\s*\(([^()]*(?:\([^()]*\)[^()]*)*)\)\s*;", src):
        name, params = m.group(1), m.group(2).strip()
        if params in ("", "void"):
            out[name] = 0
        else:
            depth, count = 0, 1
            for ch in params:
                depth += ch == "("
                depth -= ch == ")"
                count += ch == "," and depth == 0
            out[name] = count
    return out


def test_binding_signatures_match_header_prototypes():
    from paper_2604_20731_gb300 import _lib
    protos = _prototypes()
    assert set(protos) >= set(declared_functions())
    for name, (_, argtypes) in _lib.SIGNATURES.items():
        assert name in protos, name
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])


def _prototype_params():
    """name -> list of parameter declarations for every prototype."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src)
    out = {}
    for m in re.finditer(r"([a-z_][a-z0-9_]*)\s*\(([^()]*)\)\s*;", src):
        params = [p.strip() for p in m.group(2).split(",")] if m.group(2).strip() not in ("", "void") else []
        out[m.group(1)] = params
    return out


def test_binding_parameter_types_match_header():
    from paper_2604_20731_gb300 import _lib
    scalars = {"double": C.c_double, "int": C.c_int, "size_t": C.c_size_t, "int64_t": C.c_int64,
               "float": C.c_float}
    for name, params in _prototype_params().items():
        argtypes = _lib.SIGNATURES[name][1]
        assert len(params) == len(argtypes), name
        for decl, at in zip(params, argtypes):
            if "*" in decl:
                assert at is C.c_void_p or at is C.c_char_p or issubclass(at, C._Pointer), (name, decl, at)
            else:
                base = decl.replace("const ", "").split()[0]
                if base in scalars:
                    assert at is scalars[base], (name, decl, at)
                else:  # enums travel as int
                    assert at is C.c_int, (name, decl, at)


def test_binding_return_types_match_header():
    from paper_2604_20731_gb300 import _lib
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src)
    expect = {"ads_status": C.c_int, "size_t": C.c_size_t, "void": None, "const char*": C.c_char_p,
              "int": C.c_int}
    seen = 0
    for m in re.finditer(r"^\s*((?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?)\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
        ret, name = re.sub(r"\s+\*", "*", m.group(1).strip()), m.group(2)
        if name not in _lib.SIGNATURES:
            continue
        assert ret in expect, (name, ret)
        assert _lib.SIGNATURES[name][0] is expect[ret], (name, ret, _lib.SIGNATURES[name][0])
        seen += 1
    assert seen == len(_lib.SIGNATURES)


def test_struct_field_offsets_match_c(lib, tmp_path):
    """Every field of every ctypes structure sits at the offset a C compiler
    gives the header's struct (offsetof), and every struct has the C size."""
    import shutil
    import subprocess
    from paper_2604_20731_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [_lib.ads_source, _lib.ads_params, _lib.crvpinn_params, _lib.ads_allocator,
               _lib.hybrid_params, _lib.hybrid_stats, _lib.ads_server_config, _lib.ads_request_spec,
               _lib.ads_request_result, _lib.ads_server_stats_t]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "adsgb.h"', "int main(void) {"]
    expect = []
    for S in structs:
        lines.append(f'  printf("%lu\\n", (unsigned long)sizeof({S.__name__}));')
        expect.append(C.sizeof(S))
        for fname, _ in S._fields_:
            lines.append(f'  printf("%lu\\n", (unsigned long)offsetof({S.__name__}, {fname}));')
            expect.append(getattr(S, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "offsets.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "offsets"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect


def _mutate(p, crv, what):
    import math
    if what == "dim=1": p.dim = 1
    elif what == "n=1": p.n = 1
    elif what == "n 2D too large": p.n = 8193
    elif what == "n 3D too large": p.dim, p.n = 3, 513
    elif what == "n 2D FP64 strip": p.n, p.ads_dtype = 7169, 0
    elif what == "phi=0": p.phi = 0.0
    elif what == "mu_w=0": p.mu_w = 0.0
    elif what == "mu_g=nan": p.mu_g = math.nan
    elif what == "grav<0": p.grav = -1.0
    elif what == "grav=inf": p.grav = math.inf
    elif what == "grav_sign=nan": p.grav_sign = math.nan
    elif what == "n_src=9": p.n_src = 9
    elif what == "n_src=-1": p.n_src = -1
    elif what == "sigma=0": p.src[0].sigma = 0.0
    elif what == "rate<0": p.src[0].rate = -1.0
    elif what == "rate=inf": p.src[0].rate = math.inf
    elif what == "kind=2": p.src[0].kind = 2
    elif what == "ads_dtype=bf16": p.ads_dtype = 2
    elif what == "layers=3": crv.hidden_layers = 3
    elif what == "width=96": crv.width = 96
    elif what == "dtype=5": crv.dtype = 5
    elif what == "f64 width 128": crv.width, crv.dtype = 128, 0
    elif what == "act_chunks<0": crv.act_chunks = -1
    elif what == "n=2 with network": p.n = 2
    else: raise KeyError(what)


@pytest.mark.parametrize("what,code", [
    ("dim=1", 7), ("n=1", 1), ("n 2D too large", 1), ("n 3D too large", 1), ("n 2D FP64 strip", 1),
    ("phi=0", 1), ("mu_w=0", 1), ("mu_g=nan", 1), ("grav<0", 1), ("grav=inf", 1),
    ("grav_sign=nan", 1), ("n_src=9", 1), ("n_src=-1", 1), ("sigma=0", 1), ("rate<0", 1),
    ("rate=inf", 1), ("kind=2", 1), ("ads_dtype=bf16", 1), ("layers=3", 7), ("width=96", 7),
    ("dtype=5", 7), ("f64 width 128", 7), ("act_chunks<0", 1), ("n=2 with network", 1)])
def test_parameter_validation_before_any_cuda_call(lib, what, code):
    """Each refusal of the parameter check: ads_init returns its status before
    touching the GPU (K is not even looked at), and ads_hbm_estimate gives 0."""
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import make_params
    p = make_params(scn.make_scenario(2, 16), "f32")
    crv = _lib.crvpinn_params(64, 4, _lib.ADS_F32, 0)
    assert lib.ads_hbm_estimate(C.byref(p), C.byref(crv)) > 0
    _mutate(p, crv, what)
    out = C.c_void_p()
    assert lib.ads_init(C.byref(p), C.byref(crv), None, None, None, None, C.byref(out)) == code
    assert not out.value
    assert lib.ads_hbm_estimate(C.byref(p), C.byref(crv)) == 0


NULL_SWEEP = r"""
import ctypes as C, json, math
from paper_2604_20731_gb300 import _lib
lib = _lib.load()
skip = {"ads_init", "ads_init_with_allocator", "ads_hbm_estimate", "ads_status_str",
        "ads_saturation_step_noalloc", "ads_saturation_step_noalloc_status", "hybrid_step_batch"}
res = {}
for name, (rt, args) in _lib.SIGNATURES.items():
    if (name in skip or name.startswith("ads_server_") or name.startswith("ads_degree_")
            or name.startswith("ads_map_") or not args
            or args[0] is not C.c_void_p):
        continue
    vals = [None]
    for a in args[1:]:
        vals.append(0.0 if a is C.c_double else (0 if a in (C.c_int, C.c_size_t, C.c_int64) else None))
    r = getattr(lib, name)(*vals)
    res[name] = r.decode() if isinstance(r, bytes) else r
# server: NULL handles and invalid configurations (checked before any CUDA call)
out = C.c_void_p()
srv = {"create_null": lib.ads_server_create(None, C.byref(out)),
       "wait_null": lib.ads_server_wait(None, 0, 1.0, None, None, None),
       "stats_null": lib.ads_server_stats(None, None),
       "submit_null": lib.ads_server_submit(None, None, None, None, None, None, None)}
for label, cfg in (("budget0", (0, 4, 2)), ("active0", (1 << 30, 0, 2)), ("streams0", (1 << 30, 4, 0)),
                   ("streams65", (1 << 30, 4, 65))):
    srv[label] = lib.ads_server_create(C.byref(_lib.ads_server_config(*cfg)), C.byref(out))
lib.ads_server_destroy(None)
# batch
hp = _lib.hybrid_params(10, 1.0, 1, 0.1, 0.05, 100, 1e-3)
arr = (C.c_void_p * 1)()
srv["batch_null"] = lib.hybrid_step_batch(None, 0, C.byref(hp), None)
srv["batch_profile_null"] = lib.hybrid_step_batch_profile(None, 2, 1, None)
srv["batch_profile_one"] = lib.hybrid_step_batch_profile((C.c_void_p * 1)(None), 1, 1, (C.c_double * 8)())
srv["batch_negative"] = lib.hybrid_step_batch(arr, -1, C.byref(hp), None)
# allocation-free step: argument checks before any CUDA call
from paper_2604_20731_gb300 import scenario as scn
from paper_2604_20731_gb300.solver import make_params
def noalloc(mut, same=False, dt=1e-3):
    p = make_params(scn.make_scenario(2, 8), "f64")
    mut(p)
    a, b = C.c_void_p(0x1000), C.c_void_p(0x2000)
    return lib.ads_saturation_step_noalloc(C.byref(p), a, None, a, a, dt, a if same else b, None)
na = {"same_in_out": noalloc(lambda p: None, same=True), "dim3": noalloc(lambda p: setattr(p, "dim", 3)),
      "f32": noalloc(lambda p: setattr(p, "ads_dtype", 1)), "n513": noalloc(lambda p: setattr(p, "n", 513)),
      "dt0": noalloc(lambda p: None, dt=0.0), "dt_inf": noalloc(lambda p: None, dt=math.inf),
      "nsrc9": noalloc(lambda p: setattr(p, "n_src", 9)), "n1": noalloc(lambda p: setattr(p, "n", 1)),
      "grav_nan": noalloc(lambda p: setattr(p, "grav", math.nan)),
      "grav_neg": noalloc(lambda p: setattr(p, "grav", -1.0)),
      "grav_sign_nan": noalloc(lambda p: setattr(p, "grav_sign", math.nan)),
      "rate_neg": noalloc(lambda p: setattr(p.src[0], "rate", -1.0)),
      "rate_inf": noalloc(lambda p: setattr(p.src[0], "rate", math.inf)),
      "sigma0": noalloc(lambda p: setattr(p.src[0], "sigma", 0.0)),
      "kind2": noalloc(lambda p: setattr(p.src[0], "kind", 2))}
na["null"] = lib.ads_saturation_step_noalloc(None, None, None, None, None, 1e-3, None, None)
# degree-p plans: refusals before any CUDA call; the steps refuse a NULL plan
def degree(mut, deg=3):
    p = make_params(scn.make_scenario(2, 8), "f64")
    mut(p)
    plan = C.c_void_p(0x1)
    rc = lib.ads_degree_plan_create(C.byref(p), deg, C.byref(plan))
    return [rc, plan.value is None]
dg = {"deg1": degree(lambda p: None, 1), "deg5": degree(lambda p: None, 5),
      "dim3": degree(lambda p: setattr(p, "dim", 3)), "f32": degree(lambda p: setattr(p, "ads_dtype", 1)),
      "n4097": degree(lambda p: setattr(p, "n", 4097)), "n1": degree(lambda p: setattr(p, "n", 1)),
      "rate_neg": degree(lambda p: setattr(p.src[0], "rate", -1.0)),
      "grav_nan": degree(lambda p: setattr(p, "grav", math.nan))}
dg["null_out"] = [lib.ads_degree_plan_create(C.byref(make_params(scn.make_scenario(2, 8), "f64")), 3, None), True]
dg["null_params"] = [lib.ads_degree_plan_create(None, 3, C.byref(C.c_void_p())), True]
dg["step_null_plan"] = [lib.ads_degree_step(None, None, None, None, None, 1e-3, None, None), True]
dg["mass_null_plan"] = [lib.ads_degree_mass(None, None, C.byref(C.c_double()), None), True]
dg["vjp_null_plan"] = [lib.ads_degree_step_vjp(None, None, None, None, None, 1e-3, None, None, None, None, None), True]
dg["coeffs_null"] = [lib.ads_degree_coeffs(None), True]
dg["project_null_plan"] = [lib.ads_degree_project(None, None, None, None), True]
dg["project_vjp_null_plan"] = [lib.ads_degree_project_vjp(None, None, None, None), True]
dg["cfl_null_plan"] = [lib.ads_degree_cfl_dt(None, None, None, None, 0.1, 0.05, 1.0, C.byref(C.c_double()), None), True]
lib.ads_degree_plan_destroy(None)
# image maps: refusals before any CUDA call (the pointers are never dereferenced)
def mp(img=0x10000, ptype=0, dim=2, shape=(8, 8, 0), flip=1, n=(4, 4, 0), mean=0, scale=1.0, off=0.0,
       out=0x20000):
    sh = None if shape is None else (C.c_int * 3)(*shape)
    nn = None if n is None else (C.c_int * 3)(*n)
    return lib.ads_map_from_image(img, ptype, dim, sh, flip, nn, mean, scale, off, out, None)
mps = {"null_img": mp(img=None), "null_out": mp(out=None), "null_shape": mp(shape=None), "null_n": mp(n=None),
       "dim1": mp(dim=1), "dim4": mp(dim=4), "n0": mp(n=(0, 4, 0)), "n65537": mp(n=(4, 65537, 0)),
       "shape0": mp(shape=(8, 0, 0)), "shape_big": mp(shape=(1 << 25, 8, 0)), "ptype2": mp(ptype=2),
       "mean2": mp(mean=2), "scale_nan": mp(scale=math.nan), "offset_inf": mp(off=math.inf),
       "overlap": mp(out=0x10000 + 128), "misaligned_f32": mp(img=0x10002),
       "misaligned_out": mp(out=0x20004), "nodes_2e31": mp(n=(65536, 65536, 0)),
       "z0_3d": mp(dim=3, shape=(8, 8, 0), n=(4, 4, 4)), "nz0_3d": mp(dim=3, shape=(8, 8, 8), n=(4, 4, 0))}
print(json.dumps({"ctx": res, "server": srv, "noalloc": na, "degree": dg, "maps": mps}))
"""


def test_null_handles_and_refused_arguments_before_any_cuda_call(lib):
    """Every ctx-taking entry point refuses a NULL context with
    ADS_ERR_INVALID_ARG; the server and the allocation-free step refuse bad
    arguments before touching the GPU.  Run in a child process: a crash fails
    the test instead of the session."""
    import json
    import subprocess
    import sys
    # no GPU visible to the child: a check that slipped ends in a CUDA error
    # (a status the test rejects), never in a kernel launch on fake pointers
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", NULL_SWEEP], cwd=ROOT, capture_output=True, text=True,
                         timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    ctx = r["ctx"]
    assert ctx.pop("ads_last_error") == "null context"
    assert ctx.pop("ads_destroy") is None
    assert len(ctx) >= 20
    assert all(v == 1 for v in ctx.values()), {k: v for k, v in ctx.items() if v != 1}
    assert all(v == 1 for v in r["server"].values()), r["server"]
    na = r["noalloc"]
    assert na["dim3"] == 7 and na["f32"] == 7
    refused = ("same_in_out", "n513", "dt0", "dt_inf", "nsrc9", "n1", "grav_nan", "grav_neg",
               "grav_sign_nan", "rate_neg", "rate_inf", "sigma0", "kind2", "null")
    assert all(na[k] == 1 for k in refused), na
    dg = r["degree"]
    assert dg.pop("dim3") == [7, True] and dg.pop("f32") == [7, True]
    assert dg.pop("coeffs_null") == [0, True]
    assert all(v == [1, True] for v in dg.values()), dg
    assert all(v == 1 for v in r["maps"].values()), r["maps"]
