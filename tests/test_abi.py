"""The C-ABI library builds, loads, exports what include/rid.h declares, and the
ctypes structure matches the C layout.  No compute call is made here."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rid.h")
LIB = os.path.join(ROOT, "paper_2405_16076_gb300", "librid.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2405_16076_gb300.build import build
        build()
    return ctypes.CDLL(LIB)


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rid_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["rid_init", "rid_ingest", "rid_finalize", "rid_error_estimate", "rid_destroy",
                 "rid_config_default", "rid_last_error", "rid_get_basis", "rid_get_state",
                 "rid_reset", "rid_sync", "rid_n_obs"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rid_\w+)", out))
    assert set(declared_functions()) <= exported


@pytest.mark.parametrize("struct", ["rid_config", "rid_log_record"])
def test_ctypes_layout_matches_c(lib, struct):
    from paper_2405_16076_gb300 import rid
    cls = getattr(rid, struct)
    fields = [f for f, _ in cls._fields_]
    cname = {"lambda_": "lambda"}                   # a Python keyword, renamed in the binding
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"rid.h\"\nint main(void){\n"
    src += f'printf("%zu\\n", sizeof({struct}));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof({struct}, {cname.get(f, f)}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(cls)
    for f, off in zip(fields, vals[1:]):
        assert getattr(cls, f).offset == off, f


def test_defaults_and_validation_without_device(lib):
    from paper_2405_16076_gb300 import rid
    cfg = rid.rid_config()
    assert rid.rid_config_default(ctypes.byref(cfg)) == rid.RID_OK
    assert abs(cfg.c1 - 1 / 6) < 1e-15 and abs(cfg.c2 - 1 / 3) < 1e-15
    assert cfg.eps == 0.5 and cfg.delta == 0.05 and cfg.omega_kind == rid.RID_OMEGA_RADEMACHER
    h = ctypes.c_void_p()
    cfg.m, cfg.k, cfg.s, cfg.h = 100, 10, 5, 0          # s <= k is rejected before any device call
    assert rid.rid_init(ctypes.byref(h), ctypes.byref(cfg)) == rid.RID_EINVAL
    assert b"s must" in rid.rid_last_error(None)
    cfg.s, cfg.c1, cfg.c2 = 43, 0.4, 0.3                 # c1 < c2 required (Algorithm 8)
    assert rid.rid_init(ctypes.byref(h), ctypes.byref(cfg)) == rid.RID_EINVAL


def test_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2405_16076_gb300 import rid
    with pytest.raises(rid.RIDError) as e:
        rid.OnlineRID(m=1000, k=5, s=23, h=12)
    assert e.value.code == rid.RID_ENOLIB


def test_config_check_matches_init_validation(lib):
    from paper_2405_16076_gb300 import rid
    assert rid.rid_config_check(None) == rid.RID_EINVAL
    cfg = rid.make_config(100, 10, 43, 12)
    assert rid.rid_config_check(ctypes.byref(cfg)) == rid.RID_OK
    cfg.s = 10                                           # s <= k
    assert rid.rid_config_check(ctypes.byref(cfg)) == rid.RID_EINVAL
    assert b"s must" in rid.rid_last_error(None)
    cfg = rid.make_config(100, 10, 43, 12, dtype="f64", sketch="bf16x2")
    assert rid.rid_config_check(ctypes.byref(cfg)) == rid.RID_EINVAL
    assert b"FP32" in rid.rid_last_error(None)
    cfg = rid.make_config(100, 10, 43, 12, group_max=65)
    assert rid.rid_config_check(ctypes.byref(cfg)) == rid.RID_EINVAL
    cfg = rid.make_config(100, 10, 43, 12, batch_sms=-1)
    assert rid.rid_config_check(ctypes.byref(cfg)) == rid.RID_EINVAL
    assert b"batch_sms" in rid.rid_last_error(None)
    cfg = rid.make_config(100, 10, 43, 12, ingest_ctas=-1)
    assert rid.rid_config_check(ctypes.byref(cfg)) == rid.RID_EINVAL
    assert b"ingest_ctas" in rid.rid_last_error(None)


def test_autotune_argument_checks_without_device(lib):
    import torch
    from paper_2405_16076_gb300 import rid
    dummy = ctypes.c_void_p(16)                          # never dereferenced: every check fails first
    us = ctypes.c_double()
    cfg = rid.make_config(1000, 10, 43, 12)
    assert rid.rid_autotune(None, dummy, 1000, 8, ctypes.byref(us)) == rid.RID_EINVAL
    assert rid.rid_autotune(ctypes.byref(cfg), None, 1000, 8, ctypes.byref(us)) == rid.RID_EINVAL
    assert rid.rid_autotune(ctypes.byref(cfg), dummy, 1000, 0, ctypes.byref(us)) == rid.RID_EINVAL
    assert b"ncols" in rid.rid_last_error(None)
    assert rid.rid_autotune(ctypes.byref(cfg), dummy, 999, 8, ctypes.byref(us)) == rid.RID_EINVAL
    bad = rid.make_config(1000, 10, 9, 12)
    assert rid.rid_autotune(ctypes.byref(bad), dummy, 1000, 8, ctypes.byref(us)) == rid.RID_EINVAL
    assert b"s must" in rid.rid_last_error(None)
    rc = rid.rid_autotune(ctypes.byref(cfg), dummy, 1000, 8, ctypes.byref(us))
    if torch.cuda.is_available():
        assert rc == rid.RID_EINVAL                      # a host address is refused before any launch
    else:
        assert rc == rid.RID_ENOLIB
    assert cfg.group_max == 0                            # nothing written on failure


def test_log_calls_reject_null_handles(lib):
    from paper_2405_16076_gb300 import rid
    assert rid.rid_log_enable(None, 4) == rid.RID_EINVAL
    assert rid.rid_get_log(None, None, 0, None) == rid.RID_EINVAL


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_plain_c_client_links_and_validates(lib, compiler, std):
    """The boundary is usable from C (and C++) alone: a program includes rid.h, links
    librid.so, checks a configuration and reads the error text; rid_init reports RID_ENOLIB
    without a device (or succeeds with one)."""
    src = r'''
#include <stdio.h>
#include "rid.h"
int main(void) {
  rid_config c;
  if (rid_config_default(&c) != RID_OK) return 10;
  c.m = 4096; c.k = 20; c.s = 83; c.h = 30;
  if (rid_config_check(&c) != RID_OK) return 11;
  c.s = 20;
  if (rid_config_check(&c) != RID_EINVAL) return 12;
  if (!rid_last_error(NULL) || !rid_last_error(NULL)[0]) return 13;
  c.s = 83;
  rid_handle* h = NULL;
  int rc = rid_init(&h, &c);
  if (rc == RID_OK) { rid_destroy(h); printf("device\n"); return 0; }
  if (rc != RID_ENOLIB || h != NULL) return 14;
  printf("no device\n");
  return 0;
}
'''
    libdir = os.path.dirname(LIB)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "client.c")
        exe = os.path.join(d, "client")
        open(c, "w").write(src)
        lang = ["-x", "c++"] if compiler == "g++" else []
        subprocess.run([compiler, std, "-Wall", "-Werror", *lang, "-I", os.path.join(ROOT, "include"), c,
                        "-L", libdir, "-lrid", f"-Wl,-rpath,{libdir}", "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() in ("device", "no device")


def test_tuning_cache_file_parsing():
    """The autotuner's cache (csrc/tune_cache.h, host C++ only): the last valid line of a key wins;
    other keys, malformed lines and out-of-range values are skipped; stores append a line."""
    src = r'''
#include <stdio.h>
#include "tune_cache.h"
int main(int argc, char** argv) {
  const char* path = argv[1];
  int g = -1, c = -1; double us = 0;
  if (rid::tune_cache_lookup(path, "missing", 64, &g, &c, &us)) return 10;
  if (!rid::tune_cache_lookup(path, "devA|m5", 64, &g, &c, &us)) return 11;
  printf("%d %d %.3f\n", g, c, us);
  if (rid::tune_cache_lookup(path, "devB|m5", 16, &g, &c, &us)) return 12;   // its group 32 > 16
  rid::tune_cache_store(path, "devC|m7", 8, 101, 12.5);
  if (!rid::tune_cache_lookup(path, "devC|m7", 64, &g, &c, &us)) return 13;
  printf("%d %d %.3f\n", g, c, us);
  if (rid::tune_cache_lookup("/nonexistent/dir/cache", "devA|m5", 64, &g, &c, &us)) return 14;
  return 0;
}
'''
    csrc = os.path.join(ROOT, "paper_2405_16076_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "cache.txt")
        with open(cache, "w") as f:
            f.write("devA|m5 16 0 3.5\n"
                    "devB|m5 32 50 2.0\n"
                    "garbage line\n"
                    "devA|m5 0 0 1.0\n"            # group out of range: skipped
                    "devA|m5 64 -3 1.0\n"          # negative CTA count: skipped
                    "devA|m5 32 76 2.25\n"         # the last valid line for devA
                    "devA|m5 8 0 -1\n")            # non-positive time: skipped
        c = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-I", csrc, c, "-o", exe], check=True)
        r = subprocess.run([exe, cache], capture_output=True, text=True)
        assert r.returncode == 0, (r.returncode, r.stdout)
        assert r.stdout.split("\n")[:2] == ["32 76 2.250", "8 101 12.500"]
        assert open(cache).read().splitlines()[-1] == "devC|m7 8 101 12.5"


def test_fault_injection_parsing_and_countdown():
    """RID_FAULT_INJECT (csrc/fault_inject.h, host C++ only): only "alloc:<n>" with n >= 1 arms
    the allocation countdown, and then exactly the n-th allocation fails, once; only "wait:<n>"
    with 1 <= n <= 2^22 sets a pipeline-wait limit."""
    src = r'''
#include <stdio.h>
#include "fault_inject.h"
int main(void) {
  const char* off[] = {0, "", "alloc:", "alloc:0", "alloc:-2", "alloc:3x", "free:3", "ALLOC:3"};
  for (const char* v : off)
    if (rid::parse_fault_inject(v) != 0) return 10;
  if (rid::parse_fault_inject("alloc:1") != 1 || rid::parse_fault_inject("alloc:37") != 37) return 11;
  rid::AllocCountdown c;
  for (int i = 0; i < 5; ++i) if (c.next_fails()) return 12;          // disarmed
  c.arm(3);
  const bool seq[6] = {c.next_fails(), c.next_fails(), c.next_fails(), c.next_fails(), c.next_fails(),
                       c.next_fails()};
  if (seq[0] || seq[1] || !seq[2] || seq[3] || seq[4] || seq[5]) return 13;
  c.arm(0);
  if (c.next_fails()) return 14;
  const char* woff[] = {0, "", "wait:", "wait:0", "wait:-1", "wait:4194305", "wait:2x", "alloc:3"};
  for (const char* v : woff)
    if (rid::parse_wait_inject(v) != 0) return 15;
  if (rid::parse_wait_inject("wait:1") != 1 || rid::parse_wait_inject("wait:4194304") != 4194304u) return 16;
  if (rid::parse_fault_inject("wait:5") != 0) return 17;
  printf("ok\n");
  return 0;
}
'''
    csrc = os.path.join(ROOT, "paper_2405_16076_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-I", csrc, c, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout)
