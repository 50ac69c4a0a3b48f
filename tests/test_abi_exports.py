"""The C-ABI library loads and exports every entry point declared in include/*.h
(no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(precode_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2304_12745_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "precode_solve" in names and "precode_plan" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2304_12745_gb300 import capi
    capi.LIB.precode_status_str.restype = ctypes.c_char_p
    assert capi.LIB.precode_status_str(0) == b"ok"
    assert capi.LIB.precode_status_str(1) == b"invalid argument"


def test_instance_descriptor_packing_matches_abi_layout():
    import numpy as np
    from paper_2304_12745_gb300.precoder import inst_table
    t = inst_table([0, 4096], [2, 4098], [0, 8], [64, 256], [8, 32]).numpy()
    assert t.shape == (2, 4) and t.dtype == np.int64
    raw = t.view(np.int32).reshape(2, 8)
    assert list(t[1, :3]) == [4096, 4098, 8]
    assert list(raw[0, 6:]) == [64, 8] and list(raw[1, 6:]) == [256, 32]


C_PROGRAM = r"""
#include <pthread.h>
#include <stdio.h>
#include <string.h>
#include "precode.h"

/* precode_last_error() is per thread: two threads fail differently, each reads its own */
static void* fail_plan(void* arg) {
  precode_shape_t shape = {64, 8};
  precode_desc_t d;
  precode_plan_t plan;
  int i, ok = 1;
  (void)arg;
  memset(&d, 0, sizeof d);
  d.mode = PRECODE_LAYER_PROJ;
  d.n_shapes = 1;
  d.shapes = &shape;
  d.max_instances = 1;
  for (i = 0; i < 2000; ++i) {
    precode_plan(&d, &plan);
    ok &= strstr(precode_last_error(), "T out of range") != NULL;
  }
  return ok ? arg : NULL;
}
static void* fail_errors(void* arg) {
  int i, ok = 1;
  for (i = 0; i < 2000; ++i) {
    precode_plan_errors(NULL, NULL);
    ok &= strstr(precode_last_error(), "precode_plan_errors") != NULL;
  }
  return ok ? arg : NULL;
}

int main(void) {
  precode_plan_t plan = (precode_plan_t)0;
  precode_shape_t shape = {64, 8};
  precode_desc_t d;
  if (precode_plan(NULL, &plan) != PRECODE_EINVAL) return 1;
  memset(&d, 0, sizeof d);
  d.mode = PRECODE_LAYER_PROJ;
  d.T = 0; /* out of range: rejected before any device call */
  d.n_shapes = 1;
  d.shapes = &shape;
  d.max_instances = 16;
  if (precode_plan(&d, &plan) != PRECODE_EINVAL || plan != NULL) return 2;
  if (strstr(precode_last_error(), "T out of range") == NULL) return 3;
  d.T = 10;
  d.mode = 7;
  if (precode_plan(&d, &plan) != PRECODE_EINVAL) return 4;
  if (strcmp(precode_status_str(PRECODE_OK), "ok") != 0) return 5;
  if (sizeof(precode_inst_t) != 32 || sizeof(precode_shape_t) != 8) return 6;
  /* every entry point rejects a NULL handle or descriptor before touching a device */
  {
    float f[16];
    int32_t fl[2];
    uint64_t u = 0;
    char buf[64];
    precode_inst_t tbl[1];
    precode_job_t job;
    precode_result_t res;
    precode_serve_stats_t st;
    precode_server_t srv = (precode_server_t)0;
    memset(&job, 0, sizeof job);
    memset(tbl, 0, sizeof tbl);
    if (precode_plan_destroy(NULL) != PRECODE_EINVAL) return 10;
    if (precode_solve(NULL, 64, 8, 1, f, f, 0, f, NULL, f, f, f, fl, NULL) != PRECODE_EINVAL) return 11;
    if (precode_solve_host(NULL, 64, 8, 1, f, f, 0, f, NULL, f, f, f, fl) != PRECODE_EINVAL) return 12;
    if (precode_solve_varlen(NULL, 1, tbl, f, f, f, NULL, f, f, f, fl, NULL) != PRECODE_EINVAL) return 13;
    if (precode_train_step(NULL, 64, 8, 1, f, f, 0, f, NULL, 1.f, f, f, NULL, fl, NULL) != PRECODE_EINVAL)
      return 14;
    if (precode_solve_varlen_static(NULL, 1, tbl, f, f, f, NULL, f, f, f, fl, NULL) != PRECODE_EINVAL)
      return 15;
    if (precode_serve_create(NULL, &srv) != PRECODE_EINVAL || srv != NULL) return 16;
    if (precode_serve_submit(NULL, &job, &u) != PRECODE_EINVAL) return 17;
    if (precode_serve_poll(NULL, 1, &res) != PRECODE_EINVAL) return 18;
    if (precode_serve_wait(NULL, 1, 0, &res) != PRECODE_EINVAL) return 19;
    if (precode_serve_stats(NULL, &st) != PRECODE_EINVAL) return 20;
    if (precode_serve_reset_stats(NULL) != PRECODE_EINVAL) return 21;
    if (precode_serve_channel_create(NULL, 64, 8, 1, f, &u) != PRECODE_EINVAL) return 22;
    if (precode_serve_channel_destroy(NULL, 1) != PRECODE_EINVAL) return 23;
    if (precode_serve_destroy(NULL) != PRECODE_EINVAL) return 24;
    if (precode_plan_errors(NULL, &u) != PRECODE_EINVAL) return 25;
    if (precode_plan_describe(NULL, 64, 8, buf, sizeof buf) != PRECODE_EINVAL) return 26;
    if (precode_plan_set_debug(NULL, 1000, 1) != PRECODE_EINVAL) return 27;
  }
  {
    pthread_t a, b;
    void *ra = NULL, *rb = NULL;
    int tag = 1;
    pthread_create(&a, NULL, fail_plan, &tag);
    pthread_create(&b, NULL, fail_errors, &tag);
    pthread_join(a, &ra);
    pthread_join(b, &rb);
    if (ra != &tag || rb != &tag) return 30;
  }
  {
    int c;
    for (c = PRECODE_OK; c <= PRECODE_ENOTFOUND; ++c)
      if (precode_status_str((precode_status_t)c) == NULL || precode_status_str((precode_status_t)c)[0] == 0)
        return 31;
  }
  puts("c-abi ok");
  return 0;
}
"""


def test_header_is_plain_c_and_library_links_from_c(tmp_path):
    """include/precode.h compiles as strict C99 with every warning an error, and a C
    program links against libprecode.so and gets PRECODE_EINVAL back from every entry
    point for NULL handles and bad descriptors, without a GPU."""
    import shutil
    import subprocess
    from paper_2304_12745_gb300 import build
    lib_path = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib_path)
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-pthread",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-l:" + os.path.basename(lib_path),
                           "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "c-abi ok", (out.returncode, out.stderr)


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the C
    compiler gives the header's struct (a mismatch would corrupt arguments silently)."""
    import json
    import shutil
    import subprocess
    from paper_2304_12745_gb300 import capi
    pairs = {"Shape": "precode_shape_t", "Desc": "precode_desc_t",
             "ServeDesc": "precode_serve_desc_t", "Job": "precode_job_t",
             "Result": "precode_result_t", "ServeStats": "precode_serve_stats_t"}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "precode.h"',
             "int main(void) {", '  printf("{");']
    first = True
    for py, c in pairs.items():
        for name, _ in getattr(capi, py)._fields_:
            lines.append(f'  printf("{"" if first else ","}\\"{py}.{name}\\": %zu", offsetof({c}, {name}));')
            first = False
        lines.append(f'  printf(",\\"{py}\\": %zu", sizeof({c}));')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    cc = shutil.which("gcc") or shutil.which("cc")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           str(src), "-o", str(exe)])
    got = json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)
    for py in pairs:
        cls = getattr(capi, py)
        assert got[py] == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert got[f"{py}.{name}"] == getattr(cls, name).offset, (py, name)


def _header_params():
    """{function: [parameter kind]} from the prototypes in include/*.h, a kind being
    'ptr' or (int|float, bytes)."""
    scalar = {"int32_t": ("int", 4), "uint32_t": ("int", 4), "int64_t": ("int", 8),
              "uint64_t": ("int", 8), "size_t": ("int", 8), "float": ("float", 4),
              "double": ("float", 8)}
    handles = {"precode_plan_t", "precode_server_t", "precode_stream_t"}
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"precode_status_t\s+(precode_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src):
            kinds = []
            for p in m.group(2).split(","):
                p = " ".join(p.split())
                if not p or p == "void":
                    continue
                ty = p.rsplit(" ", 1)[0].replace("const ", "").strip()
                if "*" in p or ty in handles:
                    kinds.append("ptr")
                else:
                    kinds.append(scalar[ty])
            out[m.group(1)] = kinds
    return out


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    if t in (ctypes.c_float, ctypes.c_double):
        return ("float", ctypes.sizeof(t))
    return ("int", ctypes.sizeof(t))


def test_binding_signatures_match_the_prototypes():
    """Each ctypes signature of the binding has the header prototype's parameter count,
    and pointer / integer / float kinds and widths, position by position."""
    from paper_2304_12745_gb300 import capi
    proto = _header_params()
    for name, args in capi._SIGS.items():
        assert name in proto, name
        assert [_ctypes_kind(a) for a in args] == proto[name], name
