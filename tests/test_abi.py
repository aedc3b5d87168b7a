"""The C ABI library loads and exports every entry point its headers declare;
argument errors are reported synchronously (no device work is issued)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hg[a-z]*_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libs():
    from paper_1907_02900_gb300 import _build
    return _build.build()


def _lib_for(header, libs):
    base = os.path.basename(header)
    return libs["libhg_datagen.so"] if base.startswith("hgd") else libs["libhg.so"]


def test_every_declared_symbol_is_exported(libs):
    headers = glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert headers
    for h in headers:
        names = _declared(h)
        assert names, h
        lib = _lib_for(h, libs)
        out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
        exported = set(re.findall(r" T (\w+)", out))
        missing = [n for n in names if n not in exported]
        assert not missing, f"{os.path.basename(h)}: not exported by {os.path.basename(lib)}: {missing}"
        dl = ctypes.CDLL(lib)
        for n in names:
            assert getattr(dl, n) is not None


def test_status_strings_and_version(libs):
    import paper_1907_02900_gb300 as hg
    lib = hg.load()
    assert b"sm_103a" in lib.hg_version()
    for code in range(8):
        assert lib.hg_status_string(code)


def test_argument_errors_return_synchronously(libs):
    import paper_1907_02900_gb300 as hg
    lib = hg.load()
    cfg = hg.make_config(hg.KEY_U32, 1 << 10)
    fake = ctypes.c_void_p(0x10000)
    # null config
    assert lib.hg_build(None, fake, None, 10, fake, fake, fake, fake, 1 << 30, None) == 1
    # bad key type / bucket count
    bad = hg.make_config(hg.KEY_U32, 1 << 10); bad.key_type = 7
    assert lib.hg_build(ctypes.byref(bad), fake, None, 10, fake, fake, fake, fake, 1 << 30, None) == 1
    bad = hg.make_config(hg.KEY_U32, 0)
    assert lib.hg_build(ctypes.byref(bad), fake, None, 10, fake, fake, fake, fake, 1 << 30, None) == 1
    bad = hg.make_config(hg.KEY_U32, (1 << 32) + 1)
    assert lib.hg_build(ctypes.byref(bad), fake, None, 10, fake, fake, fake, fake, 1 << 30, None) == 1
    # n >= 2^32
    assert lib.hg_build(ctypes.byref(cfg), fake, None, 1 << 32, fake, fake, fake, fake, 1 << 30, None) == 1
    # misaligned keys
    mis = ctypes.c_void_p(0x10004)
    assert lib.hg_build(ctypes.byref(cfg), mis, None, 10, fake, fake, fake, fake, 1 << 30, None) == 1
    # learned map without a model
    lm = hg.make_config(hg.KEY_U64, 1 << 10); lm.map = hg.MAP_LEARNED
    assert lib.hg_build(ctypes.byref(lm), fake, None, 10, fake, fake, fake, fake, 1 << 30, None) == 6
    # probe with a null table, join with a null table
    assert lib.hg_probe(ctypes.byref(cfg), None, fake, 10, fake, None) == 1
    assert lib.hg_join_count(ctypes.byref(cfg), None, None, fake, None, fake, 1 << 20, None) == 1
    tv = hg.hg_table(10, 0x30000, 0x40000, 0x50000)
    # binned probe: null workspace, q >= 2^32, misaligned queries
    assert lib.hg_probe_binned(ctypes.byref(cfg), ctypes.byref(tv), fake, 10, fake, None, 1 << 30, None) == 1
    assert lib.hg_probe_binned(ctypes.byref(cfg), ctypes.byref(tv), fake, 1 << 32, fake, fake, 1 << 30, None) == 1
    assert lib.hg_probe_binned(ctypes.byref(cfg), ctypes.byref(tv), mis, 10, fake, fake, 1 << 30, None) == 1
    # materialisation: pairs requested without output arrays; the count's follow-up likewise
    assert lib.hg_join_materialize(ctypes.byref(cfg), ctypes.byref(tv), ctypes.byref(tv), None, None, 5, fake,
                                   fake, 1 << 30, None) == 1
    assert lib.hg_join_materialize_after_count(ctypes.byref(cfg), ctypes.byref(tv), ctypes.byref(tv), None, None,
                                               5, fake, fake, 1 << 30, None) == 1
    # the no-allocation build: V1 is not offered, n >= 2^32 is refused, and a
    # plan larger than the fixed array asks for a workspace it cannot have
    v1 = hg.make_config(hg.KEY_U32, 1 << 10, algo="v1")
    assert lib.hg_build_static_scratch(ctypes.byref(v1), fake, None, 10, fake, fake, fake, None) == 7
    assert lib.hg_build_static_scratch(ctypes.byref(cfg), fake, None, 1 << 32, fake, fake, fake, None) == 1
    big = hg.make_config(hg.KEY_U32, 1 << 28)
    assert lib.hg_build_static_scratch(ctypes.byref(big), fake, None, 1 << 28, fake, fake, fake, None) == 2
    # learned map: training without keys or model, a bad key type, statistics without outputs
    assert lib.hg_learned_train(0, None, 10, 16, 4, 8, 1, 1, fake, None, fake, 1 << 30, None) == 1
    assert lib.hg_learned_train(3, fake, 10, 16, 4, 8, 1, 1, fake, None, fake, 1 << 30, None) == 1
    assert lib.hg_learned_train(1, fake, 0, 16, 4, 8, 1, 1, fake, None, fake, 1 << 30, None) == 1
    assert lib.hg_bucket_stats(ctypes.byref(cfg), fake, 10, None, fake, fake, 1 << 20, None) == 1
    assert lib.hg_learned_judge(ctypes.byref(cfg), fake, 10, 0.0, 0.0, fake, fake, 1 << 20, None, None, None) == 1
    # batched plans: no tables, 8-byte keys, a zero bucket count
    plan = ctypes.c_void_p()
    sizes = (ctypes.c_uint64 * 2)(100, 200)
    assert lib.hg_batch_plan_create(hg.KEY_U32, 0, 0, sizes, sizes, None, ctypes.byref(plan)) == 1
    assert lib.hg_batch_plan_create(hg.KEY_U64, 0, 2, sizes, sizes, None, ctypes.byref(plan)) == 7
    zero_v = (ctypes.c_uint64 * 2)(100, 0)
    assert lib.hg_batch_plan_create(hg.KEY_U32, 0, 2, sizes, sizes, zero_v, ctypes.byref(plan)) == 1
    assert not plan.value


def test_host_buffer_call_refuses_before_any_device_work(libs):
    """hg_build_probe_host checks everything the build and the probe would
    refuse before it enqueues its first copy; on a machine without a GPU the
    refusals therefore still come back as argument errors, not CUDA errors."""
    import paper_1907_02900_gb300 as hg
    lib = hg.load()
    n, q, V = 1000, 500, 1 << 10
    cfg = hg.make_config(hg.KEY_U32, V, 0, "v2")
    fake, mis = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10004)
    host = ctypes.c_void_p(0x20000)
    tv = hg.hg_table(n, 0x30000, 0x40000, 0x50000)
    ws_need = hg.build_workspace_size(cfg, n)
    pws_need = int(lib.hg_probe_workspace_size(ctypes.byref(cfg), n, q))
    assert ws_need > 0 and pws_need > 0

    def call(table=tv, d_keys=fake, d_queries=fake, ws_bytes=ws_need, pws_bytes=pws_need, d_pws=fake):
        return lib.hg_build_probe_host(ctypes.byref(cfg), host, n, host, q, host, d_keys, d_queries, fake,
                                       ctypes.byref(table), fake, ws_bytes, d_pws, pws_bytes, None)

    assert call(table=hg.hg_table(n + 1, 0x30000, 0x40000, 0x50000)) == 1   # table size differs from n
    assert call(table=hg.hg_table(n, 0x30000, 0x40004, 0x50000)) == 1       # table keys misaligned
    assert call(d_keys=mis) == 1                                            # key staging misaligned
    assert call(d_queries=ctypes.c_void_p(0)) == 1                          # no query staging buffer
    assert call(ws_bytes=ws_need - 1) == 2                                  # build workspace short
    assert call(pws_bytes=pws_need - 1) == 2                                # probe workspace short
    assert call(d_pws=mis) == 1                                             # probe workspace misaligned


def test_workspace_sizes_cover_intermediate_arrays(libs):
    import paper_1907_02900_gb300 as hg
    for kt, kb in ((hg.KEY_U32, 4), (hg.KEY_U64, 8)):
        for n, V in ((1 << 20, 1 << 20), (1 << 28, 1 << 30), (1000, 1), (5, 1 << 24)):
            sz = hg.build_workspace_size(hg.make_config(kt, V), n)
            assert sz >= n * (kb + 4), (kt, n, V)
        v1 = hg.build_workspace_size(hg.make_config(kt, 1 << 20, algo="v1"), 1 << 20)
        assert v1 >= (1 << 20) * 4


def test_probe_workspace_grows_with_the_query_count(libs):
    """The slab-grouped probe sizes every slab's binned probe by the plan of
    all queries, so a plan for fewer queries must never need more workspace."""
    import paper_1907_02900_gb300 as hg
    lib = hg.load()
    for kt in (hg.KEY_U32, hg.KEY_U64):
        for V in (1, 1000, 1 << 20, 1 << 28):
            cfg = hg.make_config(kt, V)
            prev = 0
            for q in (1, 5, 4095, 4096, 4097, 100_000, 1 << 20, (1 << 20) + 3, 1 << 24):
                sz = int(lib.hg_probe_workspace_size(ctypes.byref(cfg), 1 << 20, q))
                assert sz >= prev and sz > 0, (kt, V, q)
                prev = sz


def test_header_is_plain_c_and_links(libs, tmp_path):
    """include/hg.h is a C header: a C99 program that takes the address of
    every declared entry point compiles without warnings (-Wall -Wextra
    -pedantic -Werror) and links against libhg.so."""
    import shutil
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    header = os.path.join(ROOT, "include", "hg.h")
    names = _declared(header)
    src = tmp_path / "uses_every_entry_point.c"
    body = "\n".join(f"  fns[{i}] = (void (*)(void))&{n};" for i, n in enumerate(names))
    src.write_text(f"""#include <stdio.h>
#include "hg.h"
int main(void) {{
  void (*fns[{len(names)}])(void);
{body}
  for (unsigned i = 0; i < {len(names)}; ++i)
    if (!fns[i]) return 1;
  puts(hg_version());
  return 0;
}}
""")
    exe = str(tmp_path / "uses_every_entry_point")
    lib = libs["libhg.so"]
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(header),
                        str(src), "-o", exe, lib, "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and "sm_103a" in run.stdout, run.stdout + run.stderr
